"""Pins of the oracle's pointwise ionic models (eq. monodomain,
eq. monodomain_g_lambda; Sec. 5 model list)."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_19994_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        if line.strip() and not line.startswith("#"):
            k, v, t = line.split()
            out[k] = (float(v), float(t))
    return out


def test_hh_rest_gates_match_published(orc):
    g = _golden("hh1952_rest.txt")
    p = I.hh1952_params()
    u = O.ionic_rest(I.MODEL_HH1952, p, -75.0)
    for name, idx in (("m_inf", 1), ("h_inf", 2), ("n_inf", 3)):
        v, tol = g[name]
        assert abs(u[idx] - v) < tol, (name, u[idx], v)


def test_hh_rest_is_equilibrium(orc):
    # HH chose E_L so that the ionic current vanishes at rest with steady gates.
    p = I.hh1952_params()
    u = O.ionic_rest(I.MODEL_HH1952, p, -75.0)
    fE, lam, yinf = O.ionic_point(I.MODEL_HH1952, p, u)
    assert abs(fE[0]) < 2e-4          # uA/mm^2
    np.testing.assert_allclose(yinf[1:], u[1:], rtol=0, atol=0)
    assert np.all(lam[1:] < 0) and lam[0] == 0.0


def test_hh_removable_singularities(orc):
    # alpha_m has 0/0 at v = 25, alpha_n at v = 10; both limits are finite and
    # the rates are continuous through them (limit of x/(e^x-1) is 1).
    p = I.hh1952_params()
    for vs in (25.0, 10.0):
        vals = []
        for dv in (-1e-3, -1e-7, 0.0, 1e-7, 1e-3):
            u = np.array([-75.0 + vs + dv, 0.1, 0.5, 0.3])
            _, lam, yinf = O.ionic_point(I.MODEL_HH1952, p, u)
            vals.append(lam[1:].copy())
        vals = np.array(vals)
        assert np.all(np.isfinite(vals))
        assert np.abs(vals[1:4] - vals[2]).max() < 1e-6
        assert np.abs(vals[0] - vals[2]).max() < 1e-2


def test_gating_form_alpha_beta(orc):
    # eq. monodomain_g_lambda: Lambda_g = -(alpha+beta), w_inf = alpha/(alpha+beta);
    # hence Lambda_g (w - w_inf) = alpha (1 - w) - beta w for any w (eq. monodomain_g),
    # with alpha = -Lambda w_inf > 0 and beta = -Lambda (1 - w_inf) > 0.
    p = I.hh1952_params()
    for V in np.linspace(-100, 60, 17):
        u = np.array([V, 0.2, 0.7, 0.4])
        _, lam, yinf = O.ionic_point(I.MODEL_HH1952, p, u)
        alpha = -lam[1:] * yinf[1:]
        beta = -lam[1:] * (1 - yinf[1:])
        assert np.all(alpha > 0) and np.all(beta > 0)
        w = u[1:]
        np.testing.assert_allclose(lam[1:] * (w - yinf[1:]), alpha * (1 - w) - beta * w, rtol=1e-12, atol=1e-15)


def _hh_rate_table():
    rows = []
    for line in open(os.path.join(GOLD, "hh1952_rates.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_hh_rates_match_published_equations(orc):
    # All six rate constants of Hodgkin & Huxley (1952), eqs. (12), (13), (20),
    # (21), (23), (24), at nine depolarisations from -30 to +100 mV (golden
    # table, evaluated in the 1952 paper's own sign convention).  They are
    # recovered from the oracle's model output: alpha = -Lambda w_inf,
    # beta = -Lambda (1 - w_inf), for m, h, n in that order.  A slip in the
    # sign or offset of any rate's voltage argument changes every row but one.
    tab = _hh_rate_table()
    assert tab.shape == (9, 7)
    p = I.hh1952_params()
    for v, am, bm, ah, bh, an, bn in tab:
        u = np.array([-75.0 + v, 0.3, 0.4, 0.5])
        _, lam, yinf = O.ionic_point(I.MODEL_HH1952, p, u)
        alpha = -lam[1:] * yinf[1:]
        beta = -lam[1:] * (1 - yinf[1:])
        np.testing.assert_allclose(alpha, [am, ah, an], rtol=1e-10, err_msg=f"alpha at v={v}")
        np.testing.assert_allclose(beta, [bm, bh, bn], rtol=1e-10, err_msg=f"beta at v={v}")


def test_hh_steady_states_and_time_constants(orc):
    # w_inf = alpha/(alpha + beta) and -1/Lambda = 1/(alpha + beta) (the 1952
    # paper's n_inf, tau_n and their m, h analogues, eqs. (8)-(9) and their
    # sodium counterparts) at the tabulated depolarisations.
    tab = _hh_rate_table()
    p = I.hh1952_params()
    for v, am, bm, ah, bh, an, bn in tab:
        _, lam, yinf = O.ionic_point(I.MODEL_HH1952, p, np.array([-75.0 + v, 0.3, 0.4, 0.5]))
        a = np.array([am, ah, an])
        b = np.array([bm, bh, bn])
        np.testing.assert_allclose(yinf[1:], a / (a + b), rtol=1e-12)
        np.testing.assert_allclose(-lam[1:], a + b, rtol=1e-12)


def test_syn19_shape_and_ranges(orc):
    # Stiff gates: rates in [1e2, 1e4] /ms, sigmoid w_inf in (0, 1); Lambda zero off the gates.
    p = I.syn19_params()
    assert p.shape == (88,)
    rng = np.random.default_rng(0)
    for V in np.linspace(-100, 60, 33):
        u = np.concatenate([[V], rng.uniform(0, 1, 18)])
        fE, lam, yinf = O.ionic_point(I.MODEL_SYN19, p, u)
        assert np.all(lam[:7] == 0) and np.all(yinf[:7] == 0) and np.all(fE[7:] == 0)
        assert np.all(-lam[7:] >= 1e2) and np.all(-lam[7:] <= 1e4)
        assert np.all(yinf[7:] > 0) and np.all(yinf[7:] < 1)
    rates = p[2:72:6] * np.exp(p[3:72:6])
    assert rates.max() > 5e3 and p[2:72:6].min() < 2e2     # the range is spanned


def test_syn19_rest_is_near_equilibrium(orc):
    p = I.syn19_params()
    u = O.ionic_rest(I.MODEL_SYN19, p, -83.4)
    fE, lam, yinf = O.ionic_point(I.MODEL_SYN19, p, u)
    np.testing.assert_allclose(fE[1:7], 0.0, atol=1e-15)   # auxiliaries at steady state
    assert abs(fE[0]) / 0.01 < 0.5                           # |dV/dt| < 0.5 mV/ms
