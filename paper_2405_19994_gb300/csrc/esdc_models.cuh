// Pointwise ionic models on the device (eq. monodomain; gates in the form of
// eq. monodomain_g_lambda).  eval() returns everything at once; currents() and
// gate() return the same numbers piecewise, so that a kernel can use each gate's
// rate as soon as it is computed; currents_f() and gate_f() are the FP32
// counterparts used by the precision form.  For one mesh node u:
//   mI   = -I_ion(u)                               [uA/mm^2]
//   ha   = h_a(u)   (NA auxiliary derivatives)
//   lam  = Lambda_g(V) = -(alpha + beta)           (NG gates)
//   yinf = w_g,inf(V) = alpha/(alpha + beta)       (NG gates)
// State order in u: V, the NA auxiliaries, the NG gates.
#pragma once
#include "esdc_fmath.cuh"
#include "esdc_internal.h"

namespace esdc {

// The two polynomials of one gate in the gate table (esdc_vtab.cpp) at
// t = V - V_mid: Horner's rule, ESDC_VTAB_NC - 1 FMAs each, on the interleaved
// coefficient pairs c[k] = (b, Lambda) of t^k, b = -Lambda w_inf.
__device__ __forceinline__ void vt_poly2(const double2* __restrict__ c, double t, double& w, double& l)
{
    const double2 top = __ldg(c + ESDC_VTAB_NC - 1);
    w = top.x;
    l = top.y;
#pragma unroll
    for (int k = ESDC_VTAB_NC - 2; k >= 0; --k) {
        const double2 ck = __ldg(c + k);
        w = fma(w, t, ck.x);
        l = fma(l, t, ck.y);
    }
}

// x/(e^x - 1), removable singularity at x = 0.  |x| < 1/2: its Taylor series
// 1 - x/2 + sum_k B_2k x^2k/(2k)! (B_2k the Bernoulli numbers), truncated after
// k = 8 (the next term is below 5e-18 there), in Horner form in x^2.
// Elsewhere x / (e^x - 1) with the library's exponential and reciprocal: e^x - 1
// loses at most a factor e^(1/2)/(e^(1/2) - 1) < 2.6 in relative accuracy for
// |x| >= 1/2, about 3 ulp in all.  About 12 FP64 operations either way.
__device__ __forceinline__ double x_over_expm1(double x)
{
    // |x| < 1/2, tested on the bit pattern (an integer compare, off the FP64 pipe)
    if ((__double_as_longlong(x) & 0x7fffffffffffffffLL) < 0x3fe0000000000000LL) {
        const double x2 = x * x;
        double p = -3617.0 / 10670622842880000.0;                 // B_16/16!
        p = fma(p, x2, 1.0 / 74724249600.0);                       // B_14/14!
        p = fma(p, x2, -691.0 / 1307674368000.0);                  // B_12/12!
        p = fma(p, x2, 1.0 / 47900160.0);                          // B_10/10!
        p = fma(p, x2, -1.0 / 1209600.0);                          // B_8/8!
        p = fma(p, x2, 1.0 / 30240.0);                             // B_6/6!
        p = fma(p, x2, -1.0 / 720.0);                              // B_4/4!
        p = fma(p, x2, 1.0 / 12.0);                                // B_2/2!
        return fma(x2, p, fma(x, -0.5, 1.0));
    }
    return x * esdc_rcp(esdc_exp(x) - 1.0);
}

// FP32 versions (the precision form): x/(e^x - 1) with a Taylor branch.
__device__ __forceinline__ float x_over_expm1f(float x)
{
    if (fabsf(x) < 1e-3f) return 1.0f - x * (0.5f - x * (1.0f / 12.0f));
    return x / expm1f(x);
}

// Hodgkin & Huxley 1952, V = Vrest + v.  params: gNa, gK, gL, ENa, EK, EL, Vrest.
struct HH1952 {
    static constexpr int NS = 4, NA = 0, NG = 3;
    static constexpr int NPARAM = 7, NDERIVED = 0;
    __device__ static void eval(const double* __restrict__ mp, const double* u, double& mI,
                                double* ha, double* lam, double* yinf)
    {
        (void)ha;
        const double V = u[0], m = u[1], h = u[2], n = u[3];
        const double m3h = m * m * m * h, n2 = n * n;
        mI = -(mp[0] * m3h * (V - mp[3]) + mp[1] * n2 * n2 * (V - mp[4]) + mp[2] * (V - mp[5]));
        for (int q = 0; q < 3; ++q) gate(mp, q, V, lam[q], yinf[q]);
    }
    // -I_ion only (the currents need the gate values, not their rates).
    __device__ static void currents(const double* __restrict__ mp, const double* u, double& mI, double* ha)
    {
        (void)ha;
        const double V = u[0], m = u[1], h = u[2], n = u[3];
        const double m3h = m * m * m * h, n2 = n * n;
        mI = -(mp[0] * m3h * (V - mp[3]) + mp[1] * n2 * n2 * (V - mp[4]) + mp[2] * (V - mp[5]));
    }
    // Rates alpha, beta of gate q (0 = m, 1 = h, 2 = n) at v = V - Vrest, with the
    // library's exponential and reciprocal (about 1 ulp each) and x_over_expm1.
    __device__ static void rates(int q, double v, double& al, double& be)
    {
        if (q == 0) { al = x_over_expm1((25.0 - v) * 0.1); be = 4.0 * esdc_exp(v * (-1.0 / 18.0)); }
        else if (q == 1) { al = 0.07 * esdc_exp(v * (-0.05)); be = esdc_rcp(esdc_exp((30.0 - v) * 0.1) + 1.0); }
        else { al = 0.1 * x_over_expm1((10.0 - v) * 0.1); be = 0.125 * esdc_exp(v * (-0.0125)); }
    }
    // Lambda_g and w_g,inf of gate q (0 = m, 1 = h, 2 = n) at potential V.
    __device__ static void gate(const double* __restrict__ mp, int q, double V, double& lam, double& yinf)
    {
        double al, be;
        rates(q, V - mp[6], al, be);
        const double sum = al + be;
        lam = -sum;
        yinf = al * esdc_rcp(sum);
    }
    // The gate table (esdc_vtab.cpp), as for SYN19: the node's interval row
    // and t = V - V_mid once per node; row = nullptr: the direct rates.
    struct VCtx {
        const double* row;
        double t;
    };
    __device__ static VCtx vctx(const ModelDev& md, double V)
    {
        VCtx c{nullptr, 0.0};
        if (md.vtab) {
            const int i = __double2int_rd((V - ESDC_VTAB_VLO) * (1.0 / ESDC_VTAB_W));
            if (i >= 0 && i < ESDC_VTAB_N) {
                c.row = md.vtab + (size_t)i * ESDC_VTAB_ROW;
                c.t = V - __ldg(c.row);
            }
        }
        return c;
    }
    // Lambda_q and b_q = -Lambda_q w_inf,q (here alpha_q): the table, else the
    // direct rates.  The gate's rate is then Lambda u + b.
    __device__ static void gate_lb(const double* __restrict__ mp, const VCtx& c, int q, double V, double& lam,
                                   double& b)
    {
        if (c.row) {
            vt_poly2(reinterpret_cast<const double2*>(c.row + 2) + q * ESDC_VTAB_NC, c.t, b, lam);
            return;
        }
        double yinf;
        gate(mp, q, V, lam, yinf);
        b = -lam * yinf;
    }
    // Lambda_q and w_inf,q (diagnostics): w_inf = -b / Lambda on the table.
    __device__ static void gate(const double* __restrict__ mp, const VCtx& c, int q, double V, double& lam,
                                double& yinf)
    {
        if (c.row) {
            double b;
            gate_lb(mp, c, q, V, lam, b);
            yinf = -b / lam;
            return;
        }
        gate(mp, q, V, lam, yinf);
    }
    __device__ static void eval(const ModelDev& md, const double* u, double& mI, double* ha, double* lam,
                                double* yinf)
    {
        (void)ha;
        const VCtx c = vctx(md, u[0]);
        for (int q = 0; q < 3; ++q) gate(md.p, c, q, u[0], lam[q], yinf[q]);
        double hl[1];
        currents(md.p, u, mI, hl);
    }
    // FP32 counterparts of currents() and gate() (parameters as floats).
    __device__ static void currents_f(const float* __restrict__ mp, const float* u, float& mI, float* ha)
    {
        (void)ha;
        const float V = u[0], m = u[1], h = u[2], n = u[3];
        const float m3h = m * m * m * h, n2 = n * n;
        mI = -(mp[0] * m3h * (V - mp[3]) + mp[1] * n2 * n2 * (V - mp[4]) + mp[2] * (V - mp[5]));
    }
    __device__ static void gate_f(const float* __restrict__ mp, int q, float V, float& lam, float& yinf)
    {
        const float v = V - mp[6];
        float al, be;
        if (q == 0) { al = x_over_expm1f((25.0f - v) * 0.1f); be = 4.0f * expf(v * (-1.0f / 18.0f)); }
        else if (q == 1) { al = 0.07f * expf(v * (-0.05f)); be = 1.0f / (expf((30.0f - v) * 0.1f) + 1.0f); }
        else { al = 0.1f * x_over_expm1f((10.0f - v) * 0.1f); be = 0.125f * expf(v * (-0.0125f)); }
        const float sum = al + be;
        lam = -sum;
        yinf = al / sum;
    }
    // Derivatives for the adjoint.  d(-I_ion)/du (u = V, m, h, n) and
    // d(-I_ion)/d(gNa, gK).
    __device__ static void currents_d(const double* __restrict__ mp, const double* u, double* dmI, double* dpar)
    {
        const double V = u[0], m = u[1], h = u[2], n = u[3];
        const double m2 = m * m, n3 = n * n * n;
        dmI[0] = -(mp[0] * m2 * m * h + mp[1] * n3 * n + mp[2]);
        dmI[1] = -3.0 * mp[0] * m2 * h * (V - mp[3]);
        dmI[2] = -mp[0] * m2 * m * (V - mp[3]);
        dmI[3] = -4.0 * mp[1] * n3 * (V - mp[4]);
        dpar[0] = -m2 * m * h * (V - mp[3]);
        dpar[1] = -n3 * n * (V - mp[4]);
    }
    // Lambda, w_inf of gate q and their derivatives in V.  With f(x) = x/(e^x - 1),
    // f'(x) = f (1 - f - x)/x, or its Taylor series -1/2 + x/6 - x^3/180 near 0.
    __device__ static void gate_d(const double* __restrict__ mp, int q, double V, double& lam, double& yinf,
                                  double& dlam, double& dyinf)
    {
        const double v = V - mp[6];
        auto fprime = [](double x, double f) {
            return fabs(x) < 1e-3 ? -0.5 + x * (1.0 / 6.0 - x * x * (1.0 / 180.0)) : f * (1.0 - f - x) / x;
        };
        double al, be, dal, dbe;
        rates(q, v, al, be);                       // the forward rates, bit for bit
        if (q == 0) {
            dal = -0.1 * fprime((25.0 - v) * 0.1, al);
            dbe = be * (-1.0 / 18.0);
        } else if (q == 1) {
            dal = -0.05 * al;
            dbe = 0.1 * be * (1.0 - be);
        } else {
            const double x = (10.0 - v) * 0.1;
            dal = 0.1 * (-0.1) * fprime(x, x_over_expm1(x));
            dbe = be * (-0.0125);
        }
        const double sum = al + be;
        lam = -sum;
        yinf = al * esdc_rcp(sum);
        dlam = -(dal + dbe);
        dyinf = (dal * be - al * dbe) / (sum * sum);
    }
    // Resting state at V0: gates at w_inf(V0).
    __device__ static void rest(const double* mp, double V0, double* u)
    {
        double mI, lam[NG], yinf[NG];
        u[0] = V0; u[1] = u[2] = u[3] = 0.0;
        eval(mp, u, mI, nullptr, lam, yinf);
        for (int g = 0; g < NG; ++g) u[1 + g] = yinf[g];
    }
};

// 19-state synthetic stiff model (shape of ten Tusscher-Panfilov 2006),
// evaluated with esdc_exp / esdc_rcp and host-side reciprocals of the constant
// divisors (each differs from the IEEE quotient by about one ulp):
// V, auxiliaries a1..a6, gates g1..g12.  params (88): 12 x (Vh, k, r, ln rho,
// Vr, sr), [G_f, E_f, G_s, E_s, G_K, E_K, G_K1, G_b, E_b, c_K6], tau_1..tau_6.
//   w_inf = 1/(1 + e^{-(V-Vh)/k}),  rate = r exp(ln rho / (1 + e^{-(V-Vr)/sr}))
//   I_ion = G_f g1 g2 g3 a1 (V-E_f) + G_s g4 g5 a3 (V-E_s)
//         + G_K a2 (1 + c_K6 a6)(V-E_K) + G_K1 g7 g8 (V-E_K)
//         + G_b (g9+g10+g11+g12)/4 (V-E_b)
//   a1' = (1-g6-a1)/tau1, a2' = (g6-a2)/tau2, a3' = (1-g6-a3)/tau3,
//   a4' = (g4 g5 - a4)/tau4, a5' = (a4-a5)/tau5, a6' = (a5-a6)/tau6
struct SYN19 {
    static constexpr int NS = 19, NA = 6, NG = 12;
    // mp[88 + q] = 1/k_q, mp[100 + q] = 1/sr_q, mp[112 + l] = 1/tau_l,
    // mp[118 + q] = Vh_q/k_q, mp[130 + q] = Vr_q/sr_q, mp[142 + q] = ln r_lo,q (set on the host):
    // (Vh - V)/k = Vh/k - V/k and r_lo exp(a) = exp(a + ln r_lo) each save an FP64 operation
    static constexpr int NPARAM = 88, NDERIVED = 66;
    __device__ static void eval(const double* __restrict__ mp, const double* u, double& mI,
                                double* ha, double* lam, double* yinf)
    {
        const double V = u[0];
        const double* a = u + 1;
        const double* g = u + 7;
        const double* inv = mp + 88;
#pragma unroll
        for (int q = 0; q < 12; ++q) gate(mp, q, V, lam[q], yinf[q]);
        const double* c = mp + 72;
        const double If = c[0] * g[0] * g[1] * g[2] * a[0] * (V - c[1]);
        const double Is = c[2] * g[3] * g[4] * a[2] * (V - c[3]);
        const double IK = c[4] * a[1] * (1.0 + c[9] * a[5]) * (V - c[5]);
        const double IK1 = c[6] * g[6] * g[7] * (V - c[5]);
        const double Ib = c[7] * 0.25 * (g[8] + g[9] + g[10] + g[11]) * (V - c[8]);
        mI = -(If + Is + IK + IK1 + Ib);
        if (ha) {
            const double* itau = inv + 24;
            ha[0] = ((1.0 - g[5]) - a[0]) * itau[0];
            ha[1] = (g[5] - a[1]) * itau[1];
            ha[2] = ((1.0 - g[5]) - a[2]) * itau[2];
            ha[3] = (g[3] * g[4] - a[3]) * itau[3];
            ha[4] = (a[3] - a[4]) * itau[4];
            ha[5] = (a[4] - a[5]) * itau[5];
        }
    }
    __device__ static void currents(const double* __restrict__ mp, const double* u, double& mI, double* ha)
    {
        const double V = u[0];
        const double* a = u + 1;
        const double* g = u + 7;
        const double* c = mp + 72;
        const double If = c[0] * g[0] * g[1] * g[2] * a[0] * (V - c[1]);
        const double Is = c[2] * g[3] * g[4] * a[2] * (V - c[3]);
        const double IK = c[4] * a[1] * (1.0 + c[9] * a[5]) * (V - c[5]);
        const double IK1 = c[6] * g[6] * g[7] * (V - c[5]);
        const double Ib = c[7] * 0.25 * (g[8] + g[9] + g[10] + g[11]) * (V - c[8]);
        mI = -(If + Is + IK + IK1 + Ib);
        const double* itau = mp + 112;
        ha[0] = ((1.0 - g[5]) - a[0]) * itau[0];
        ha[1] = (g[5] - a[1]) * itau[1];
        ha[2] = ((1.0 - g[5]) - a[2]) * itau[2];
        ha[3] = (g[3] * g[4] - a[3]) * itau[3];
        ha[4] = (a[3] - a[4]) * itau[4];
        ha[5] = (a[4] - a[5]) * itau[5];
    }
    __device__ static void gate(const double* __restrict__ mp, int q, double V, double& lam, double& yinf)
    {
        const double* p = mp + 6 * q;
        const double* inv = mp + 88;
        const double* dv = mp + 118;
        yinf = esdc_rcp(1.0 + esdc_exp(fma(-V, inv[q], dv[q])));
        const double s = esdc_rcp(1.0 + esdc_exp(fma(-V, inv[12 + q], dv[12 + q])));
        lam = -esdc_exp(fma(p[3], s, dv[24 + q]));
    }
    // The gate table (esdc_vtab.cpp): a node's interval row and t = V - V_mid,
    // computed once per node for all twelve gates; row = nullptr (no table, or
    // V outside [ESDC_VTAB_VLO, ESDC_VTAB_VLO + ESDC_VTAB_N ESDC_VTAB_W)) selects
    // the direct evaluation.  A NaN V stays NaN either way.
    struct VCtx {
        const double* row;
        double t;
    };
    __device__ static VCtx vctx(const ModelDev& md, double V)
    {
        VCtx c{nullptr, 0.0};
        if (md.vtab) {
            const int i = __double2int_rd((V - ESDC_VTAB_VLO) * (1.0 / ESDC_VTAB_W));
            if (i >= 0 && i < ESDC_VTAB_N) {
                c.row = md.vtab + (size_t)i * ESDC_VTAB_ROW;
                c.t = V - __ldg(c.row);
            }
        }
        return c;
    }
    // Lambda_q and b_q = -Lambda_q w_inf,q of gate q: two polynomials
    // (2 (ESDC_VTAB_NC - 1) FMAs) on the table, else the direct formulas (about
    // 35 FP64 operations).  The gate's rate is then Lambda u + b.
    __device__ static void gate_lb(const double* __restrict__ mp, const VCtx& c, int q, double V, double& lam,
                                   double& b)
    {
        if (c.row) {
            vt_poly2(reinterpret_cast<const double2*>(c.row + 2) + q * ESDC_VTAB_NC, c.t, b, lam);
            return;
        }
        double yinf;
        gate(mp, q, V, lam, yinf);
        b = -lam * yinf;
    }
    // Lambda_q and w_inf,q (diagnostics): w_inf = -b / Lambda on the table.
    __device__ static void gate(const double* __restrict__ mp, const VCtx& c, int q, double V, double& lam,
                                double& yinf)
    {
        if (c.row) {
            double b;
            gate_lb(mp, c, q, V, lam, b);
            yinf = -b / lam;
            return;
        }
        gate(mp, q, V, lam, yinf);
    }
    __device__ static void eval(const ModelDev& md, const double* u, double& mI, double* ha, double* lam,
                                double* yinf)
    {
        const VCtx c = vctx(md, u[0]);
#pragma unroll
        for (int q = 0; q < 12; ++q) gate(md.p, c, q, u[0], lam[q], yinf[q]);
        double hl[NA];
        currents(md.p, u, mI, ha ? ha : hl);
    }
    __device__ static void currents_f(const float* __restrict__ mp, const float* u, float& mI, float* ha)
    {
        const float V = u[0];
        const float* a = u + 1;
        const float* g = u + 7;
        const float* c = mp + 72;
        const float If = c[0] * g[0] * g[1] * g[2] * a[0] * (V - c[1]);
        const float Is = c[2] * g[3] * g[4] * a[2] * (V - c[3]);
        const float IK = c[4] * a[1] * (1.0f + c[9] * a[5]) * (V - c[5]);
        const float IK1 = c[6] * g[6] * g[7] * (V - c[5]);
        const float Ib = c[7] * 0.25f * (g[8] + g[9] + g[10] + g[11]) * (V - c[8]);
        mI = -(If + Is + IK + IK1 + Ib);
        const float* itau = mp + 112;
        ha[0] = ((1.0f - g[5]) - a[0]) * itau[0];
        ha[1] = (g[5] - a[1]) * itau[1];
        ha[2] = ((1.0f - g[5]) - a[2]) * itau[2];
        ha[3] = (g[3] * g[4] - a[3]) * itau[3];
        ha[4] = (a[3] - a[4]) * itau[4];
        ha[5] = (a[4] - a[5]) * itau[5];
    }
    __device__ static void gate_f(const float* __restrict__ mp, int q, float V, float& lam, float& yinf)
    {
        const float* p = mp + 6 * q;
        const float* inv = mp + 88;
        yinf = 1.0f / (1.0f + expf((p[0] - V) * inv[q]));
        const float s = 1.0f / (1.0f + expf((p[4] - V) * inv[12 + q]));
        lam = -p[2] * expf(p[3] * s);
    }
    __device__ static void rest(const double* mp, double V0, double* u)
    {
        double mI, lam[NG], yinf[NG];
        for (int s = 0; s < NS; ++s) u[s] = 0.0;
        u[0] = V0;
        eval(mp, u, mI, nullptr, lam, yinf);
        for (int q = 0; q < NG; ++q) u[7 + q] = yinf[q];
        const double g6 = yinf[5];
        u[1] = 1.0 - g6;
        u[2] = g6;
        u[3] = 1.0 - g6;
        u[4] = yinf[3] * yinf[4];
        u[5] = u[4];
        u[6] = u[4];
    }
};

}  // namespace esdc
