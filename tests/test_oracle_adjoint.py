"""Pins of the oracle's discrete adjoint (oracle/adjoint.py): every component
of dL/dsigma, dL/dg_Na, dL/dg_K and dL/dy0 against central differences of the
oracle's own forward map (orc_sweep.c, eq. prec_picard with eq. def_P and
eq. def_C, Sec. 3.1), on 3x3 and 6x5 Hodgkin-Huxley sheets with a
conductivity field.  The loss is linear in the sensor traces, so a central
difference carries only its O(eps^2) truncation and the forward map's
rounding."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.adjoint import HHFieldAdjoint
from paper_2405_19994_gb300 import inputs as I

NSTEPS = 6


def _case(nx, ny, seed):
    wl = I.hh_field_sheet(max(nx, ny))
    wl = wl.with_mesh(nx, ny, 1)
    wl.sigma_field = I.lognormal_field(nx, ny, 1, seed=seed, corr=1.5)
    rng = np.random.default_rng(seed)
    m = O.Monodomain(wl, solver=O.SOLVE_DENSE)
    y0 = m.init_state()
    y0[0] += rng.normal(0.0, 5.0, wl.n_nodes)         # a few mV off rest, so diffusion acts
    sens = np.sort(rng.choice(wl.n_nodes, size=min(4, wl.n_nodes), replace=False))
    wts = rng.normal(size=(NSTEPS, len(sens)))
    return wl, y0, sens, wts


def _loss(wl, y0, sens, wts, sigma=None, params=None):
    w = wl.with_mesh(wl.nx, wl.ny, wl.nz)
    w.sigma_field = wl.sigma_field if sigma is None else sigma
    w.params = wl.params if params is None else params
    adj = HHFieldAdjoint(O.Monodomain(w, solver=O.SOLVE_DENSE))
    tr, _ = adj.traces(y0, 0.0, w.dt, w.M, w.K, NSTEPS, sens)
    return float(np.sum(wts * tr))


def _grads(wl, y0, sens, wts):
    adj = HHFieldAdjoint(O.Monodomain(wl, solver=O.SOLVE_DENSE))
    return adj.sensor_gradients(y0, 0.0, wl.dt, wl.M, wl.K, NSTEPS, sens, wts)


@pytest.mark.parametrize("nx,ny,seed", [(3, 3, 11), (6, 5, 12)])
def test_adjoint_matches_central_differences_every_component(orc, nx, ny, seed):
    wl, y0, sens, wts = _case(nx, ny, seed)
    gsig, gna, gk, gy0 = _grads(wl, y0, sens, wts)
    sig = wl.sigma_field
    # conductivity field, node by node
    fd = np.empty(wl.n_nodes)
    for p in range(wl.n_nodes):
        e = 1e-5 * sig[p]
        sp, sm = sig.copy(), sig.copy()
        sp[p] += e
        sm[p] -= e
        fd[p] = (_loss(wl, y0, sens, wts, sigma=sp) - _loss(wl, y0, sens, wts, sigma=sm)) / (2 * e)
    assert np.abs(fd).max() > 0
    np.testing.assert_allclose(gsig, fd, rtol=0, atol=2e-7 * np.abs(fd).max())
    # maximal conductances
    for k, g in ((0, gna), (1, gk)):
        p = wl.params.copy()
        e = 1e-6 * p[k]
        pp, pm = p.copy(), p.copy()
        pp[k] += e
        pm[k] -= e
        f = (_loss(wl, y0, sens, wts, params=pp) - _loss(wl, y0, sens, wts, params=pm)) / (2 * e)
        assert abs(g - f) <= 2e-7 * abs(f), (k, g, f)
    # initial state, every state of every node
    for s, e in ((0, 1e-4), (1, 1e-6), (2, 1e-6), (3, 1e-6)):
        for p in range(wl.n_nodes):
            yp, ym = y0.copy(), y0.copy()
            yp[s, p] += e
            ym[s, p] -= e
            f = (_loss(wl, yp, sens, wts) - _loss(wl, ym, sens, wts)) / (2 * e)
            scale = max(np.abs(gy0[s]).max(), 1e-12)
            assert abs(gy0[s, p] - f) <= 2e-6 * scale, (s, p, gy0[s, p], f)


def test_conductivity_derivative_of_the_quadratic_form(orc):
    # d(lam^T A v)/d sigma_p: the face-sum formula of the adjoint against
    # central differences of the oracle's conductivity operator (linear in sigma)
    wl = I.hh_field_sheet(5).with_mesh(5, 4, 1)
    wl.sigma_field = I.lognormal_field(5, 4, 1, seed=3, corr=1.5)
    rng = np.random.default_rng(2)
    lam, v = rng.normal(size=20), rng.normal(size=20)
    adj = HHFieldAdjoint(O.Monodomain(wl, solver=O.SOLVE_DENSE))
    got = adj.dsig(lam, v)
    for p in range(20):
        out = []
        for sgn in (1, -1):
            w = wl.with_mesh(5, 4, 1)
            w.sigma_field = wl.sigma_field.copy()
            w.sigma_field[p] += sgn * 0.01
            out.append(lam @ O.Monodomain(w, solver=O.SOLVE_DENSE).conductivity(v))
        assert abs(got[p] - (out[0] - out[1]) / 0.02) < 1e-12 * (1 + abs(got[p]))


@pytest.mark.parametrize("K,dt", [(1, 0.1), (3, 0.05)])
def test_step_adjoint_full_state(orc, K, dt):
    # One step, a linear loss on every state of every node (gates included):
    # here the set-up's dependence on Lambda_n = Lambda(V_n) -- through
    # a_ij(dt Lambda_n) and phi_1(d_j dt Lambda_n) -- carries a large part of
    # dL/dV_n, which sensor losses on V over short runs hardly see.
    wl = I.hh_field_sheet(3).with_mesh(3, 3, 1)
    wl.sigma_field = I.lognormal_field(3, 3, 1, seed=21, corr=1.5)
    rng = np.random.default_rng(21)
    m = O.Monodomain(wl, solver=O.SOLVE_DENSE)
    y0 = m.init_state()
    y0[0] += rng.uniform(-20.0, 40.0, wl.n_nodes)
    W = rng.normal(size=y0.shape)
    adj = HHFieldAdjoint(m)
    acc = {"sig": np.zeros(wl.n_nodes), "gNa": 0.0, "gK": 0.0}
    gy = adj.step_vjp(y0, 0.3, dt, wl.M, K, W, acc)

    def L(y):
        return float(np.sum(W * m.step(y, 0.3, dt, wl.M, K)[0]))

    for s, e in ((0, 1e-4), (1, 1e-6), (2, 1e-6), (3, 1e-6)):
        for p in range(wl.n_nodes):
            yp, ym = y0.copy(), y0.copy()
            yp[s, p] += e
            ym[s, p] -= e
            f = (L(yp) - L(ym)) / (2 * e)
            assert abs(gy[s, p] - f) <= 1e-7 * max(np.abs(gy[s]).max(), 1e-12), (s, p, gy[s, p], f)
