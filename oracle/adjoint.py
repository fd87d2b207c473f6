"""Discrete adjoint of the oracle's HSDC step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; the product path never does.

What it differentiates: the oracle's own forward map, one HSDC time step of
the Hodgkin-Huxley monodomain problem with a per-node conductivity field
(Sec. 3.1), K sweeps with no stop test, in the non-recursive form that
``orc_sweep.c`` implements:

  set-up (frozen for the step, eq. def_ode_esdc, eq. def_C):
    Lambda_n = Lambda(y_n),  a_ij = a_ij(dt Lambda_n),  phi1_j = phi_1(d_j dt Lambda_n)
  g(y)     = f_I(y) + f_E(t_j, y) + f_e(y) + Lambda_n (y_n - y)            eq. def_g
  Ex_j(u)  = f_E(t_{j-1}, u) + phi1_j (f_e(u) + Lambda_n (y_n - u))
  E_j(Y)   = f_I(Y_j) + Ex_j(Y_{j-1})                                      eq. def_P
  sweep Y^k -> Y^{k+1} (eq. prec_picard with P of eq. def_P, C of eq. def_C),
  rows i = 1..M in order, Yn_0 = y_n:
    X_i   = Ex_i(Yn_{i-1})
    rhs_i = y_n + dt sum_j a_ij g(Y^k_j) + dt sum_{j<i} d_j (f_I(Yn_j) + X_j - E_j(Y^k))
            + dt d_i (X_i - E_i(Y^k))
    Yn_i  = S_i^{-1} rhs_i,   S_i = I - dt d_i f_I   (an implicit solve on the V row)
  from Y^0 = 1 (x) y_n; y_{n+1} = Y^K_M.

The reverse sweep runs these assignments backwards (reverse-mode
differentiation written out by hand, no tape library):
  * every pointwise term through its vector-Jacobian product;
  * the solve through S_i^{-T} = S_i^{-1} (f_I is symmetric) and the
    conductivity derivative of lambda^T A v, which per node p is
    -(1/(2h^2)) sum_{q in nbr(p)} (lambda_p - lambda_q)(v_p - v_q)
    for (A v)_p = (1/h^2) sum_q (sigma_p + sigma_q)/2 (v_q - v_p);
  * the set-up through d a_ij/dz = sum_k c_i^{k+1} w_j^{k-1} phi_k'(c_i z) and
    phi_k'(x) = phi_k(x) - k phi_{k+1}(x) (App. A's representation and the
    derivative of phi_k's integral definition), with phi_k from its series;
  * the Hodgkin-Huxley rates' voltage derivatives by complex-step
    differentiation of the rate formulas (exact to rounding, no cancellation).
The forward iterates Y^k of a step come from the C oracle itself (one sweep per
call from the previous iterate), so the map differentiated is exactly the
oracle's.  Gradients: dL/dsigma per node, dL/dg_Na, dL/dg_K and dL/dy_0 for a
loss of V at sensor nodes after every step.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O

_H = 1e-20          # complex-step size


def _x_over_expm1(x):
    """x / (e^x - 1) with its removable point, complex-safe: the Bernoulli
    series sum_k B_k x^k / k! below |x| = 0.1 (terms to x^10), the quotient
    above."""
    x = np.asarray(x)
    small = np.abs(x) < 0.1
    xs = np.where(small, x, 0)
    b = [1.0, -0.5, 1.0 / 12, 0.0, -1.0 / 720, 0.0, 1.0 / 30240, 0.0, -1.0 / 1209600, 0.0, 1.0 / 47900160]
    ser = np.zeros_like(xs)
    for c in reversed(b):
        ser = ser * xs + c
    xl = np.where(small, 1.0, x)
    return np.where(small, ser, xl / np.expm1(xl))


def _hh_rates(V, p):
    """alpha, beta of (m, h, n) in the rest-shifted 1952 convention (the
    oracle's model, orc_model.c): 3 x [N] arrays each, complex-safe."""
    v = V - p[6]
    am = _x_over_expm1((25.0 - v) / 10.0)
    bm = 4.0 * np.exp(-v / 18.0)
    ah = 0.07 * np.exp(-v / 20.0)
    bh = 1.0 / (np.exp((30.0 - v) / 10.0) + 1.0)
    an = 0.1 * _x_over_expm1((10.0 - v) / 10.0)
    bn = 0.125 * np.exp(-v / 80.0)
    return np.array([am, ah, an]), np.array([bm, bh, bn])


def _lam_yinf(V, p):
    a, b = _hh_rates(V, p)
    return -(a + b), a / (a + b)


def _lam_yinf_dV(V, p):
    """Lambda_g(V), w_inf,g(V) and their V-derivatives (complex step)."""
    lam, yinf = _lam_yinf(V, p)
    lc, yc = _lam_yinf(V + 1j * _H, p)
    return lam, yinf, lc.imag / _H, yc.imag / _H


def _phi_series(x, kmax):
    """phi_k(x) = sum_m x^m/(m+k)!, k = 1..kmax, elementwise ([kmax, ...])."""
    x = np.asarray(x, np.float64)
    if np.abs(x).max(initial=0.0) > 2.0:
        raise ValueError("phi series used for |x| <= 2 only")
    out = []
    for k in range(1, kmax + 1):
        s = np.zeros_like(x)
        for m in range(40, -1, -1):
            s = s * x + 1.0 / math.factorial(m + k)
        out.append(s)
    return np.array(out)


class HHFieldAdjoint:
    """The oracle's step map for an HH workload with a conductivity field, and
    its discrete adjoint.  ``mono`` is an ``oracle.Monodomain`` built on that
    workload (exact or 1e-15 CG solves)."""

    def __init__(self, mono: O.Monodomain):
        wl = mono.wl
        if wl.model != 0 or getattr(wl, "sigma_field", None) is None:
            raise ValueError("the adjoint covers Hodgkin-Huxley with a conductivity field")
        self.m = mono
        self.wl = wl
        self.N, self.ns = mono.N, mono.ns
        self.p = np.array(wl.params, np.float64)
        self.sig = np.asarray(wl.sigma_field, np.float64).reshape(-1)
        self.ichiCm = 1.0 / (wl.chi * wl.Cm)
        self.ih2 = 1.0 / wl.h ** 2
        self.shape = (wl.nz, wl.ny, wl.nx)

    # ------------------------------------------------------------ pointwise pieces
    def fI(self, u):
        out = np.zeros_like(u)
        out[0] = self.m.conductivity(u[0]) * self.ichiCm
        return out

    def I_ion(self, u):
        V, mm, hh, nn = u
        gNa, gK, gL, ENa, EK, EL = self.p[:6]
        return gNa * mm ** 3 * hh * (V - ENa) + gK * nn ** 4 * (V - EK) + gL * (V - EL)

    def stim(self, t):
        wl = self.wl
        s = np.zeros(self.shape)
        for b in range(len(wl.amp)):
            x0, x1, y0, y1, z0, z1 = wl.boxes[b]
            if wl.t_on[b] <= t < wl.t_off[b]:
                s[z0:z1, y0:y1, x0:x1] += wl.amp[b]
        return s.reshape(-1)

    def fE(self, t, u):
        out = np.zeros_like(u)
        out[0] = (self.stim(t) - self.I_ion(u)) / self.wl.Cm
        return out

    def fe(self, u):
        lam, yinf = _lam_yinf(u[0], self.p)
        out = np.zeros_like(u)
        out[1:] = lam * (u[1:] - yinf)
        return out

    # ------------------------------------------------------------ their vector-Jacobian products
    def dsig(self, lam, v):
        """d(lam^T A v)/d sigma_p = -(1/(2h^2)) sum_{q in nbr(p)} (lam_p - lam_q)(v_p - v_q)."""
        L = lam.reshape(self.shape)
        W = v.reshape(self.shape)
        g = np.zeros(self.shape)
        for ax in range(3):
            if self.shape[ax] < 2:
                continue
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, -1)
            hi[ax] = slice(1, None)
            lo, hi = tuple(lo), tuple(hi)
            t = (L[lo] - L[hi]) * (W[lo] - W[hi])        # face between the two nodes
            g[lo] += t
            g[hi] += t
        return (-0.5 * self.ih2 * g).reshape(-1)

    def vjp_fI(self, u, w, ubar, acc):
        ubar[0] += self.m.conductivity(w[0]) * self.ichiCm       # A is symmetric
        acc["sig"] += self.dsig(w[0], u[0]) * self.ichiCm

    def vjp_fE(self, u, w, ubar, acc):
        V, mm, hh, nn = u
        gNa, gK, gL, ENa, EK, EL = self.p[:6]
        c = -w[0] / self.wl.Cm
        ubar[0] += c * (gNa * mm ** 3 * hh + gK * nn ** 4 + gL)
        ubar[1] += c * 3.0 * gNa * mm ** 2 * hh * (V - ENa)
        ubar[2] += c * gNa * mm ** 3 * (V - ENa)
        ubar[3] += c * 4.0 * gK * nn ** 3 * (V - EK)
        acc["gNa"] += float(np.sum(c * mm ** 3 * hh * (V - ENa)))
        acc["gK"] += float(np.sum(c * nn ** 4 * (V - EK)))

    def vjp_fe(self, u, w, ubar):
        lam, yinf, dlam, dyinf = _lam_yinf_dV(u[0], self.p)
        ubar[1:] += lam * w[1:]
        ubar[0] += np.sum((dlam * (u[1:] - yinf) - lam * dyinf) * w[1:], axis=0)

    # ------------------------------------------------------------ one step
    def _setup(self, yn, dt, M):
        c = O.radau_nodes(M)
        d = np.diff(c)
        wF = O.fornberg_weights(M, c)                      # wF[k, j] = w_j^k
        lam_g = _lam_yinf(yn[0], self.p)[0]                # [3, N]
        lam_n = np.zeros_like(yn)
        lam_n[1:] = lam_g
        # a_ij(z) = sum_k c_i^k w_j^{k-1} phi_k(c_i z) and its z-derivative,
        # elementwise for z = dt Lambda_n, k = 1..M (App. A)
        a = np.zeros((M, M) + yn.shape)
        da = np.zeros((M, M) + yn.shape)
        z = dt * lam_n
        for i in range(M):
            ci = c[i + 1]
            ph = _phi_series(ci * z, M + 1)                 # [M+1, ns, N]
            for j in range(M):
                for k in range(1, M + 1):
                    a[i, j] += ci ** k * wF[k - 1, j] * ph[k - 1]
                    da[i, j] += ci ** (k + 1) * wF[k - 1, j] * (ph[k - 1] - k * ph[k])
        phi1 = np.zeros((M,) + yn.shape)
        dphi1 = np.zeros((M,) + yn.shape)
        for j in range(M):
            ph = _phi_series(d[j] * z, 2)
            phi1[j] = ph[0]
            dphi1[j] = ph[0] - ph[1]
        return c, d, lam_n, a, da, phi1, dphi1

    def _iterates(self, yn, t, dt, M, K):
        """Y^0 .. Y^K of the step from the C oracle ([K+1, M, ns, N])."""
        Ys = [np.broadcast_to(yn, (M,) + yn.shape).copy()]
        for _ in range(K):
            _, _, col, _ = self.m.step(yn, t, dt, M, 1, want_colloc=True, colloc_in=Ys[-1])
            Ys.append(col)
        return np.array(Ys)

    def step_vjp(self, yn, t, dt, M, K, ybar_next, acc):
        """Adjoint of y_{n+1} = step(y_n): returns dL/dy_n given dL/dy_{n+1},
        and adds the parameter gradients to acc (keys sig, gNa, gK)."""
        c, d, lam_n, a, da, phi1, dphi1 = self._setup(yn, dt, M)
        Ys = self._iterates(yn, t, dt, M, K)
        tj = t + c * dt
        g_solve = [dt * d[i] * self.ichiCm for i in range(M)]
        ynbar = np.zeros_like(yn)
        lambar = np.zeros_like(yn)
        abar = np.zeros_like(a)
        phibar = np.zeros_like(phi1)

        def vjp_Ex(j, u, Xbar, ubar):
            # Ex_j(u) = f_E(t_{j-1}, u) + phi1_j (f_e(u) + Lambda_n (y_n - u)); j 0-based
            self.vjp_fE(u, Xbar, ubar, acc)
            Zbar = phi1[j] * Xbar
            self.vjp_fe(u, Zbar, ubar)
            ubar -= lam_n * Zbar
            ynbar[:] += lam_n * Zbar
            lambar[:] += (yn - u) * Zbar
            phibar[j] += (self.fe(u) + lam_n * (yn - u)) * Xbar

        def vjp_g(j, u, Gbar, ubar):
            self.vjp_fI(u, Gbar, ubar, acc)
            self.vjp_fE(u, Gbar, ubar, acc)
            self.vjp_fe(u, Gbar, ubar)
            ubar -= lam_n * Gbar
            ynbar[:] += lam_n * Gbar
            lambar[:] += (yn - u) * Gbar

        Ybar = np.zeros((M,) + yn.shape)                   # adjoint of Y^K
        Ybar[M - 1] = ybar_next
        for k in range(K - 1, -1, -1):                     # sweep k: Y^k -> Y^{k+1}
            Yk, Yk1 = Ys[k], Ys[k + 1]
            prev = lambda i, Y: yn if i == 0 else Y[i - 1]  # noqa: E731  Y_{i-1} with Y_0 = y_n
            Gk = [self.fI(Yk[j]) + self.fE(tj[j + 1], Yk[j]) + self.fe(Yk[j]) + lam_n * (yn - Yk[j])
                  for j in range(M)]
            Ynbar = Ybar                                     # adjoint of Y^{k+1}, completed below
            Wbar = np.zeros((M,) + yn.shape)                 # adjoint of f_I(Yn_j) + X_j
            Xbar = np.zeros((M,) + yn.shape)
            Gbar = np.zeros((M,) + yn.shape)
            Ebar = np.zeros((M,) + yn.shape)
            for i in range(M - 1, -1, -1):
                # W_i = f_I(Yn_i) + X_i: its adjoint is complete (only rows > i use it)
                self.vjp_fI(Yk1[i], Wbar[i], Ynbar[i], acc)
                Xbar[i] += Wbar[i]
                # Yn_i = S_i^{-1} rhs_i (V row; the other rows are the identity)
                rbar = Ynbar[i].copy()
                rbar[0] = self.m.solve_A(g_solve[i], Ynbar[i][0])
                acc["sig"] += g_solve[i] * self.dsig(rbar[0], Yk1[i][0])
                # rhs_i = y_n + dt sum_j a_ij G_j + dt sum_{j<i} d_j (W_j - E_j) + dt d_i (X_i - E_i)
                ynbar[:] += rbar
                for j in range(M):
                    Gbar[j] += dt * a[i, j] * rbar
                    abar[i, j] += dt * Gk[j] * rbar
                for j in range(i):
                    Wbar[j] += dt * d[j] * rbar
                    Ebar[j] -= dt * d[j] * rbar
                Xbar[i] += dt * d[i] * rbar
                Ebar[i] -= dt * d[i] * rbar
                # X_i = Ex_i(Yn_{i-1})
                ubar = ynbar if i == 0 else Ynbar[i - 1]
                vjp_Ex(i, prev(i, Yk1), Xbar[i], ubar)
            # G_j = g(Y^k_j) and E_j = f_I(Y^k_j) + Ex_j(Y^k_{j-1})
            Ybar = np.zeros((M,) + yn.shape)
            for j in range(M):
                vjp_g(j, Yk[j], Gbar[j], Ybar[j])
                self.vjp_fI(Yk[j], Ebar[j], Ybar[j], acc)
                vjp_Ex(j, prev(j, Yk), Ebar[j], ynbar if j == 0 else Ybar[j - 1])
        ynbar += Ybar.sum(axis=0)                          # Y^0 = 1 (x) y_n
        # set-up: a_ij(dt Lambda_n), phi1_j(d_j dt Lambda_n), Lambda_n = Lambda(V_n)
        lambar += dt * np.einsum("ijsn,ijsn->sn", abar, da)
        for j in range(M):
            lambar += phibar[j] * d[j] * dt * dphi1[j]
        _, _, dlam, _ = _lam_yinf_dV(yn[0], self.p)
        ynbar[0] += np.sum(dlam * lambar[1:], axis=0)
        return ynbar

    # ------------------------------------------------------------ many steps, sensor loss
    def traces(self, y0, t0, dt, M, K, nsteps, sens):
        """V at the sensor nodes after every step ([nsteps, nsens]) and the
        states y_0 .. y_{nsteps-1} the steps start from."""
        y = np.array(y0, np.float64).reshape(self.ns, self.N)
        out, states = [], []
        t = t0
        for _ in range(nsteps):
            states.append(y)
            y, _, _, _ = self.m.step(y, t, dt, M, K)
            out.append(y[0][sens])
            t += dt
        return np.array(out), states

    def sensor_gradients(self, y0, t0, dt, M, K, nsteps, sens, dtraces):
        """Gradients of a loss L(traces) with dL/dtraces = dtraces [nsteps,
        nsens]: (dL/dsigma [N], dL/dg_Na, dL/dg_K, dL/dy0 [ns, N])."""
        _, states = self.traces(y0, t0, dt, M, K, nsteps, sens)
        acc = {"sig": np.zeros(self.N), "gNa": 0.0, "gK": 0.0}
        ybar = np.zeros((self.ns, self.N))
        for n in range(nsteps - 1, -1, -1):
            np.add.at(ybar[0], sens, dtraces[n])
            ybar = self.step_vjp(states[n], t0 + n * dt, dt, M, K, ybar, acc)
        return acc["sig"], acc["gNa"], acc["gK"], ybar
