"""Generate the constants of the binary64 exponential used by the fit (ksdf_exp.cuh).

The fit needs exp(-lambda r^2) to binary64 accuracy.  Its argument is carried in units of ln2 / 2^16:
e = (2^16 / ln2) lambda r^2, so that the value is 2^(-e / 2^16).  With n = round(e) = 2^16 m + 2^8 a + b
(0 <= a, b < 256) and r = e - n (|r| <= 1/2),
    2^(-e / 2^16) = 2^-m * T1[a] * T2[b] * exp(-C1 r),   T1[a] = 2^(-a/256),  T2[b] = 2^(-b/65536),
and exp(-C1 r) = 1 - C1 r + C1^2 r^2 / 2 to within 3e-17 (C1 = ln2 / 2^16, |C1 r| <= 5.3e-6).  This is a
two-level table method in the spirit of P. T. P. Tang ("Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989) with a table fine enough for a
second-degree polynomial.  This script computes the tables and constants with 60-digit decimal arithmetic
and prints them; run it to reproduce the literals in ksdf_exp.cuh.
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def ln2():
    # ln 2 = sum_{k>=1} 1 / (k 2^k)
    s, t, k = Decimal(0), Decimal(1) / 2, 1
    while True:
        term = t / k
        if term < Decimal(10) ** -58:
            break
        s += term
        t /= 2
        k += 1
    return s


def exp_dec(x: Decimal) -> Decimal:
    # Taylor series; |x| < 1 here
    s, t, k = Decimal(1), Decimal(1), 1
    while abs(t) > Decimal(10) ** -58:
        t = t * x / k
        s += t
        k += 1
    return s


def to_double(d: Decimal) -> float:
    return float(d)  # correctly rounded (Python converts the decimal string exactly)


def main():
    L = ln2()
    c1 = L / 65536
    print("// ln2 / 2^16, (ln2 / 2^16)^2 / 2, 2^16 / ln2")
    print("constexpr double kExpC1 = %s;" % to_double(c1).hex())
    print("constexpr double kExpC2 = %s;" % to_double(c1 * c1 / 2).hex())
    print("constexpr double kExpQ16PerNat = %s;" % to_double(Decimal(65536) / L).hex())
    for name, den in (("kExpT1", 256), ("kExpT2", 65536)):
        print("// %s[j] = 2^(-j/%d), j = 0..255" % (name, den))
        vals = [to_double(exp_dec(-Decimal(j) * L / den)).hex() for j in range(256)]
        for i in range(0, 256, 4):
            print("    " + ", ".join(vals[i:i + 4]) + ",")


if __name__ == "__main__":
    main()
