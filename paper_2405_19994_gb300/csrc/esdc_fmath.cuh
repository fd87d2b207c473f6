// FP64 exponential and reciprocal with few FP64-pipe operations.  On GB300
// the FP64 pipe issues about 2 operations per clock per SM (64x fewer than FP32),
// so the ionic model's exponentials and divisions set the speed of the sweep.
//
// esdc_exp: the table-driven method of P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989, with a 64-entry table:
//   x = (64 m + j) ln2/64 + r,  j in [0, 64),  |r| <= ln2/128,
//   e^x = 2^m * 2^(j/64) * e^r,   e^r = 1 + q(r),  q = Taylor degree 5
// (|r|^6/720 < 3.6e-17, below half an ulp).  k = 64 m + j = rint(64 x / ln2)
// comes from the round-to-nearest "add 1.5*2^52" trick; ln2/64 is split into a
// 29-bit head and a tail so k * head is exact (|k| < 2^17).  2^m is applied by adding m to
// the exponent field (an integer operation).  Error: about 1 ulp.
// |x| < 512 takes the fast path (the range test is an integer test on the
// high word); elsewhere arguments below -707 return 0 (results < 1e-307),
// above 709.78 return +inf, NaN returns NaN.  Cost: 10 FP64 operations, 1 table
// load.
//
// esdc_rcp: 1/d by two Newton steps r <- r + r (1 - d r) from the FP32
// reciprocal (relative error 2^-22 -> 2^-44 -> rounding), about 1 ulp, for
// 2^-99 <= |d| < 2^100 (an integer test on the exponent field); other values
// (0, tiny, huge, inf, NaN) use the IEEE division.  Cost: 4 FP64 operations and
// two conversions.
#pragma once
#include <cstdint>

namespace esdc {

// 2^(j/64), j = 0..63, rounded to nearest double (computed at 60 digits).
static __device__ const double g_exp2_table[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0,
};

static __device__ __noinline__ double esdc_exp_wide(double x)
{
    if (!(x >= -707.0)) return (x != x) ? x : 0.0;
    if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);
    return exp(x);
}

__device__ __forceinline__ double esdc_exp(double x)
{
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40800000) return esdc_exp_wide(x);   // |x| >= 512 or NaN
    const double kInvL = 0x1.71547652b82fep+6;           // 64 / ln 2
    const double kMagic = 0x1.8p+52;                      // 1.5 * 2^52
    const double kL1 = 0x1.62e42ff000000p-7;              // ln2/64, leading 29 bits
    const double kL2 = -0x1.718432a1b0e26p-41;            // ln2/64 - kL1
    const double t = fma(x, kInvL, kMagic);               // 1.5*2^52 + rint(64 x/ln2)
    const int k = __double2loint(t);                      // low word holds k
    const double kd = t - kMagic;
    double r = fma(-kd, kL1, x);
    r = fma(-kd, kL2, r);
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    q = q * r;                                            // e^r - 1
    const int j = k & 63;
    const long long m = (long long)((k - j) >> 6);
    const double T = __ldg(&g_exp2_table[j]);
    const double e = fma(T, q, T);                        // 2^(j/64) e^r, in [0.99, 2.02)
    return __longlong_as_double(__double_as_longlong(e) + (m << 52));
}

__device__ __forceinline__ double esdc_rcp(double d)
{
    const unsigned ex = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
    if (ex - 924u > 198u) return 1.0 / d;
    double r = (double)__frcp_rn((float)d);
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

}  // namespace esdc
