// FP64 exponential and reciprocal with few FP64-pipe operations.  On GB300
// the FP64 pipe issues about 2 operations per clock per SM (64x fewer than FP32),
// so the ionic model's exponentials and divisions set the speed of the sweep.
//
// esdc_exp: the table-driven method of P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989, with a 2048-entry table:
//   x = (2048 m + j) ln2/2048 + r,  j in [0, 2048),  |r| <= ln2/4096,
//   e^x = 2^m * 2^(j/2048) * e^r,   e^r = 1 + q(r),  q = Taylor degree 3
// (|r|^4/24 < 3.5e-17, below a third of an ulp).  k = 2048 m + j =
// rint(2048 x/ln2) comes from the round-to-nearest "add 1.5*2^52" trick;
// ln2/2048 is split into a 29-bit head and a tail so k * head is exact
// (|k| < 2^21).  2^m is applied by adding m to the exponent field (an integer
// operation).  Error: about 1 ulp.  |x| < 512 takes the fast path (the range
// test is an integer test on the high word); elsewhere arguments below -707
// return 0 (results < 1e-307), above 709.78 return +inf, NaN returns NaN.
// Cost: 8 FP64 operations and one load from a 16 KB table (esdc_exp_table.h),
// which stays in L1.
//
// esdc_rcp: 1/d from the hardware reciprocal approximation r =
// rcp.approx.ftz.f64(d) by one third-order step: with e = 1 - d r (one FMA,
// exact to first order), 1/d = r/(1 - e) = r (1 + e + e^2 + ...), so
// r + r (e + e^2) has relative error e^3 plus the final rounding (the
// truncated geometric series, the third-order member of the Newton-type
// reciprocal iterations).  About 1 ulp for 2^-99 <= |d| < 2^100 (an integer
// test on the exponent field); other values (0, tiny, huge, inf, NaN) use the
// IEEE division.  Cost: 3 FP64 operations.
#pragma once
#include <cstdint>

#include "esdc_exp_table.h"

namespace esdc {

static __device__ __noinline__ double esdc_exp_wide(double x)
{
    if (!(x >= -707.0)) return (x != x) ? x : 0.0;
    if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);
    return exp(x);
}

__device__ __forceinline__ double esdc_exp(double x)
{
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40800000) return esdc_exp_wide(x);   // |x| >= 512 or NaN
    const double kInvL = 0x1.71547652b82fep+11;          // 2048 / ln 2
    const double kMagic = 0x1.8p+52;                      // 1.5 * 2^52
    const double kL1 = 0x1.62e42ff000000p-12;             // ln2/2048, leading 29 bits
    const double kL2 = -0x1.718432a1b0e26p-46;            // ln2/2048 - kL1
    const double t = fma(x, kInvL, kMagic);               // 1.5*2^52 + rint(2048 x/ln2)
    const int k = __double2loint(t);                      // low word holds k
    const double kd = t - kMagic;
    double r = fma(-kd, kL1, x);
    r = fma(-kd, kL2, r);
    double q = fma(r, 1.0 / 6.0, 0.5);
    q = fma(q, r, 1.0);
    q = q * r;                                            // e^r - 1
    const int j = k & 2047;
    const long long m = (long long)((k - j) >> 11);
    const double T = __ldg(&g_exp2_table[j]);
    const double e = fma(T, q, T);                        // 2^(j/2048) e^r, in [0.9997, 2.0)
    return __longlong_as_double(__double_as_longlong(e) + (m << 52));
}

__device__ __forceinline__ double esdc_rcp(double d)
{
    const unsigned ex = ((unsigned)__double2hiint(d) >> 20) & 0x7ffu;
    if (ex - 924u > 198u) return 1.0 / d;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

}  // namespace esdc
