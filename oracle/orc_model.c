/*
 * orc_model.c -- pointwise ionic models for the HSDC oracle (test
 * infrastructure only; see esdc_oracle.h).
 *
 * The paper writes every ionic model in the form of eq. (monodomain):
 *   C_m V' = ... + I_stim - I_ion(V, w_a, w_g),  w_a' = h_a,
 *   w_g'   = Lambda_g(V) (w_g - w_g,inf(V)),  Lambda_g = -(alpha + beta),
 *   w_g,inf = alpha / (alpha + beta)                    (eq. monodomain_g_lambda)
 * and splits the right-hand side as f_E = (C_m^{-1}(I_stim - I_ion), h_a, 0),
 * f_e = Lambda (y - y_inf) with Lambda nonzero on the gates only (eq. def_f_IE,
 * eq. def_Lambda).  This file returns, for one mesh node u = (V, w_a, w_g):
 *   fE   = (-I_ion, h_a, 0)   (the caller forms (I_stim - I_ion)/C_m)
 *   lam  = (0, 0, Lambda_g(V))
 *   yinf = (0, 0, w_g,inf(V))
 *
 * HH1952: Hodgkin & Huxley (1952), J. Physiol. 117:500, in the convention
 * V = Vrest + v (v = depolarisation from rest, mV), rates in 1/ms.
 *   params: [gNa, gK, gL, ENa, EK, EL, Vrest]  (mS/mm^2, mV)
 *   states: [V, m, h, n]; m1 = 0, m2 = 3.
 *
 * SYN19: a seeded synthetic stiff model with the shape of ten Tusscher-
 * Panfilov 2006 (19 states: V, 6 auxiliaries, 12 gates; Sec. 5), because the
 * paper gives no TTP equations.  Each gate q has
 *   w_inf,q(V) = 1/(1 + exp(-(V - Vh_q)/k_q)),
 *   rate_q(V)  = r_q * exp(lnrho_q * s((V - Vr_q)/sr_q)),  s(u) = 1/(1+e^{-u}),
 *   Lambda_q   = -rate_q.
 * Currents (uA/mm^2):
 *   I_f  = G_f g1 g2 g3 a1 (V - E_f)            fast inward, slow inactivation a1
 *   I_s  = G_s g4 g5 a3 (V - E_s)               plateau inward
 *   I_K  = G_K a2 (1 + c_K6 a6) (V - E_K)       delayed outward
 *   I_K1 = G_K1 g7 g8 (V - E_K)                 inward rectifier
 *   I_b  = G_b (g9 + g10 + g11 + g12)/4 (V - E_b)
 * Auxiliaries (time constants tau_l, ms):
 *   a1' = ((1 - g6) - a1)/tau1   a2' = (g6 - a2)/tau2   a3' = ((1 - g6) - a3)/tau3
 *   a4' = (g4 g5 - a4)/tau4      a5' = (a4 - a5)/tau5   a6' = (a5 - a6)/tau6
 *   params: [12 x (Vh, k, r, lnrho, Vr, sr)] then
 *           [G_f, E_f, G_s, E_s, G_K, E_K, G_K1, G_b, E_b, c_K6] then
 *           [tau1..tau6]   -> 72 + 10 + 6 = 88 values.
 */
#include "esdc_oracle.h"
#include <math.h>

int orc_mono_nstate(int model) { return model == ORC_HH1952 ? 4 : 19; }
int orc_mono_ngate(int model)  { return model == ORC_HH1952 ? 3 : 12; }

/* x / (e^x - 1), with its removable singularity at x = 0 (Taylor branch). */
static double x_over_expm1(double x)
{
    if (fabs(x) < 1e-6) return 1.0 - 0.5 * x + x * x / 12.0;
    return x / expm1(x);
}

static void hh_rates(const double* mp, double V, double* alpha, double* beta)
{
    double v = V - mp[6];
    alpha[0] = x_over_expm1((25.0 - v) / 10.0);                 /* alpha_m */
    beta[0]  = 4.0 * exp(-v / 18.0);                            /* beta_m  */
    alpha[1] = 0.07 * exp(-v / 20.0);                           /* alpha_h */
    beta[1]  = 1.0 / (exp((30.0 - v) / 10.0) + 1.0);            /* beta_h  */
    alpha[2] = 0.1 * x_over_expm1((10.0 - v) / 10.0);           /* alpha_n */
    beta[2]  = 0.125 * exp(-v / 80.0);                          /* beta_n  */
}

static void hh_point(const double* mp, const double* u, double* fE, double* lam, double* yinf)
{
    double V = u[0], m = u[1], h = u[2], n = u[3];
    double gNa = mp[0], gK = mp[1], gL = mp[2], ENa = mp[3], EK = mp[4], EL = mp[5];
    double I_ion = gNa * m * m * m * h * (V - ENa) + gK * n * n * n * n * (V - EK) + gL * (V - EL);
    double a[3], b[3];
    hh_rates(mp, V, a, b);
    fE[0] = -I_ion;
    lam[0] = 0.0; yinf[0] = 0.0;
    for (int g = 0; g < 3; ++g) {
        fE[1 + g] = 0.0;
        lam[1 + g] = -(a[g] + b[g]);
        yinf[1 + g] = a[g] / (a[g] + b[g]);
    }
}

static double logistic(double x) { return 1.0 / (1.0 + exp(-x)); }

static void syn_point(const double* mp, const double* u, double* fE, double* lam, double* yinf)
{
    double V = u[0];
    const double* a = u + 1;          /* a1..a6 -> a[0..5]  */
    const double* g = u + 7;          /* g1..g12 -> g[0..11] */
    for (int q = 0; q < 12; ++q) {
        const double* p = mp + 6 * q;
        double winf = logistic((V - p[0]) / p[1]);
        double rate = p[2] * exp(p[3] * logistic((V - p[4]) / p[5]));
        lam[7 + q] = -rate;
        yinf[7 + q] = winf;
        fE[7 + q] = 0.0;
    }
    const double* c = mp + 72;
    double Gf = c[0], Ef = c[1], Gs = c[2], Es = c[3], GK = c[4], EK = c[5], GK1 = c[6],
           Gb = c[7], Eb = c[8], cK6 = c[9];
    const double* tau = mp + 82;
    double I_f  = Gf * g[0] * g[1] * g[2] * a[0] * (V - Ef);
    double I_s  = Gs * g[3] * g[4] * a[2] * (V - Es);
    double I_K  = GK * a[1] * (1.0 + cK6 * a[5]) * (V - EK);
    double I_K1 = GK1 * g[6] * g[7] * (V - EK);
    double I_b  = Gb * 0.25 * (g[8] + g[9] + g[10] + g[11]) * (V - Eb);
    fE[0] = -(I_f + I_s + I_K + I_K1 + I_b);
    fE[1] = ((1.0 - g[5]) - a[0]) / tau[0];
    fE[2] = (g[5] - a[1]) / tau[1];
    fE[3] = ((1.0 - g[5]) - a[2]) / tau[2];
    fE[4] = (g[3] * g[4] - a[3]) / tau[3];
    fE[5] = (a[3] - a[4]) / tau[4];
    fE[6] = (a[4] - a[5]) / tau[5];
    for (int s = 0; s < 7; ++s) { lam[s] = 0.0; yinf[s] = 0.0; }
}

void orc_ionic_point(int model, const double* mp, const double* u,
                     double* fE, double* lam, double* yinf)
{
    if (model == ORC_HH1952) hh_point(mp, u, fE, lam, yinf);
    else syn_point(mp, u, fE, lam, yinf);
}

/* Initial state: V0, gates at w_inf(V0), auxiliaries at their V0 steady state. */
void orc_ionic_rest(int model, const double* mp, double V0, double* u)
{
    int ns = orc_mono_nstate(model);
    double fE[19], lam[19], yinf[19];
    for (int s = 0; s < ns; ++s) u[s] = 0.0;
    u[0] = V0;
    orc_ionic_point(model, mp, u, fE, lam, yinf);
    for (int s = ns - orc_mono_ngate(model); s < ns; ++s) u[s] = yinf[s];
    if (model == ORC_SYN19) {
        const double* g = u + 7;
        u[1] = 1.0 - g[5];
        u[2] = g[5];
        u[3] = 1.0 - g[5];
        u[4] = g[3] * g[4];
        u[5] = u[4];
        u[6] = u[5];
    }
}
