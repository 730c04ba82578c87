"""Generate the constants of the binary64 exponential used by the fit (ksdf_exp.cuh).

The method is the table-driven exponential of P. T. P. Tang ("Table-driven implementation of the
exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989):
    x = (32 m + j) ln2/32 + r,  |r| <= ln2/64,   exp(x) = 2^m * 2^(j/32) * exp(r).
The library uses 256 table entries: x = (256 m + j) ln2/256 + r, |r| <= ln2/512.  This script computes,
with 60-digit decimal arithmetic, ln 2 / 256 split into a head with its low 24 bits zero (so n * head is
exact for |n| < 2^24) and a tail, 256 / ln 2, and 2^(j/256) for j < 256 rounded to binary64.  Run it to
reproduce the literals in ksdf_exp.cuh.
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


def to_double(d: Decimal) -> float:
    return float(d)  # correctly rounded (Python converts the decimal string exactly)


def main():
    T = 256
    L = ln2()
    l32 = L / T
    head = float(l32)
    import struct

    bits = struct.unpack("<Q", struct.pack("<d", head))[0] & ~((1 << 24) - 1)
    head = struct.unpack("<d", struct.pack("<Q", bits))[0]
    tail = to_double(l32 - Decimal(head))
    inv = to_double(Decimal(T) / L)
    print("// ln2/256 head, tail; 256/ln2")
    print("constexpr double kLn2_TabHi = %s;  // %r" % (head.hex(), head))
    print("constexpr double kLn2_TabLo = %s;  // %r" % (tail.hex(), tail))
    print("constexpr double kInvLn2_Tab = %s;  // %r" % (inv.hex(), inv))
    print("// 2^(j/256), j = 0..255")
    vals = []
    for j in range(T):
        v = to_double((Decimal(2) ** (Decimal(j) / T)))
        vals.append(v.hex())
    for i in range(0, T, 4):
        print("    " + ", ".join(vals[i:i + 4]) + ",")


if __name__ == "__main__":
    main()
