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
    # hence Lambda_g (w - w_inf) = alpha (1 - w) - beta w for any w (eq. monodomain_g).
    # Check the identity by recovering alpha = -Lambda w_inf, beta = -Lambda (1 - w_inf).
    p = I.hh1952_params()
    for V in np.linspace(-100, 60, 17):
        u = np.array([V, 0.2, 0.7, 0.4])
        _, lam, yinf = O.ionic_point(I.MODEL_HH1952, p, u)
        alpha = -lam[1:] * yinf[1:]
        beta = -lam[1:] * (1 - yinf[1:])
        assert np.all(alpha > 0) and np.all(beta > 0)
        v = V + 75.0
        np.testing.assert_allclose(beta[0], 4.0 * np.exp(-v / 18.0), rtol=1e-10)   # recovery through 1 - w_inf cancels digits
        np.testing.assert_allclose(alpha[1], 0.07 * np.exp(-v / 20.0), rtol=1e-10)   # recovery through 1 - w_inf cancels digits
        np.testing.assert_allclose(beta[2], 0.125 * np.exp(-v / 80.0), rtol=1e-10)   # recovery through 1 - w_inf cancels digits


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
