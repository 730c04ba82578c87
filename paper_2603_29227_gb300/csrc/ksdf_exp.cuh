// ksdf_exp.cuh -- binary64 exp(x) for x <= 0 used to build the GP kernel matrix in the fit.
//
// Table-driven method of P. T. P. Tang (ACM TOMS 15(2), 1989):
//   n = round(x * 32 / ln2),  r = x - n ln2/32 (two-step, head exact),  |r| <= ln2/64 ~ 0.0109,
//   exp(x) = 2^(n div 32) * 2^((n mod 32)/32) * (1 + p(r)),  p(r) = r + r^2/2! + ... + r^7/7!
// (Taylor tail; truncation below 4e-18 for |r| <= 0.0109), so the result is within a few ulp.  About 11
// FP64 operations instead of a general-purpose exp; valid for -708 <= x <= 0 (the caller zeroes kernel
// entries far below that).  Constants from gen_exp_consts.py (60-digit decimal arithmetic).
#pragma once

namespace ksdf {

constexpr double kLn2_32Hi = 0x1.62e42fe000000p-6;
constexpr double kLn2_32Lo = 0x1.f473de6af278fp-35;
constexpr double kInvLn2_32 = 0x1.71547652b82fep+5;
constexpr double kRoundShift = 0x1.8p52;  // adding 1.5 * 2^52 rounds to an integer in the low bits

__constant__ double kExp2Frac32[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0,
};

// exp(x) for -708 <= x <= 0; `tab` is kExp2Frac32 (or a shared-memory copy of it)
__device__ __forceinline__ double exp_neg64(double x, const double* tab) {
  const double t = fma(x, kInvLn2_32, kRoundShift);
  const int n = __double2loint(t);
  const double dn = t - kRoundShift;
  double r = fma(-dn, kLn2_32Hi, x);
  r = fma(-dn, kLn2_32Lo, r);
  double p = fma(r, 1.0 / 5040.0, 1.0 / 720.0);
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p * r, r, r);  // exp(r) - 1
  const double tj = tab[n & 31];
  const double y = fma(tj, p, tj);
  const int m = n >> 5;  // floor(n / 32)
  return __hiloint2double(__double2hiint(y) + (m << 20), __double2loint(y));
}

}  // namespace ksdf
