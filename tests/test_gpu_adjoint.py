"""The differentiation form: the library's discrete adjoint of the HSDC step
(esdc_adjoint_*) against central finite differences of the GPU forward map and
of the oracle's forward map, for the gradient of a sensor misfit with respect
to the conductivity field, g_Na, g_K and the initial state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
import paper_2405_19994_gb300 as P  # noqa: E402
from paper_2405_19994_gb300 import esdc as E  # noqa: E402
from paper_2405_19994_gb300 import inputs as I  # noqa: E402

NSTEPS = 30
EPS = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    P.lib()


@pytest.fixture(scope="module")
def case():
    wl = I.hh_field_sheet(16)
    rng = np.random.default_rng(41)
    sens = np.sort(rng.choice(wl.n_nodes, size=8, replace=False)).astype(np.int32)
    s = P.Solver.from_workload(wl, M_max=wl.M)
    y0 = s.new_state()
    s.init_state(y0, wl.V0)
    # target: another conductivity field and perturbed conductances
    tgt_sig = I.lognormal_field(16, 16, 1, seed=6)
    p = wl.params.copy()
    p[0] *= 1.05
    p[1] *= 0.95
    target = run_gpu(s, wl, tgt_sig, p, y0, sens)
    return wl, s, y0, sens, target


def run_gpu(s, wl, sig, params, y0, sens, want_ckpt=False):
    s.set_params(params)
    s.set_conductivity_field(sig)
    y = y0.clone()
    sd = torch.from_numpy(sens).cuda()
    tr = torch.empty((NSTEPS, len(sens)), dtype=torch.float64, device="cuda")
    ck = torch.empty((NSTEPS, s.n_state, s.ld), dtype=torch.float64, device="cuda")
    s.adjoint_forward(y, 0.0, wl.dt, wl.M, wl.K, NSTEPS, sd, tr, ck)
    assert s.residual()[0] == 0
    torch.cuda.synchronize()
    return (tr.cpu().numpy(), ck) if want_ckpt else tr.cpu().numpy()


def loss(tr, target):
    return 0.5 * float(((tr - target) ** 2).sum())


def gradients(case):
    wl, s, y0, sens, target = case
    tr, ck = run_gpu(s, wl, wl.sigma_field, wl.params, y0, sens, want_ckpt=True)
    dtr = torch.from_numpy(tr - target).cuda()
    gsig, gpar, gy0 = s.adjoint_backward(ck, 0.0, wl.dt, wl.M, wl.K, NSTEPS, torch.from_numpy(sens).cuda(), dtr,
                                         want_y0=True)
    torch.cuda.synchronize()
    return tr, gsig.cpu().numpy(), gpar, gy0


def test_adjoint_conductivity_field_vs_finite_differences(case):
    wl, s, y0, sens, target = case
    tr, gsig, _, _ = gradients(case)
    assert loss(tr, target) > 0
    d = wl.sigma_field * np.random.default_rng(3).normal(size=wl.n_nodes)
    Lp = loss(run_gpu(s, wl, wl.sigma_field + EPS * d, wl.params, y0, sens), target)
    Lm = loss(run_gpu(s, wl, wl.sigma_field - EPS * d, wl.params, y0, sens), target)
    fd = (Lp - Lm) / (2 * EPS)
    ad = float(gsig @ d)
    assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)


@pytest.mark.parametrize("k", [0, 1])
def test_adjoint_conductances_vs_finite_differences(case, k):
    wl, s, y0, sens, target = case
    tr, _, gpar, _ = gradients(case)
    p = wl.params.copy()
    h = EPS * p[k]
    pp, pm = p.copy(), p.copy()
    pp[k] += h
    pm[k] -= h
    fd = (loss(run_gpu(s, wl, wl.sigma_field, pp, y0, sens), target)
          - loss(run_gpu(s, wl, wl.sigma_field, pm, y0, sens), target)) / (2 * h)
    assert abs(gpar[k] - fd) <= 1e-5 * abs(fd), (k, gpar[k], fd)


def test_adjoint_initial_state_vs_finite_differences(case):
    wl, s, y0, sens, target = case
    _, _, _, gy0 = gradients(case)
    d = torch.zeros_like(y0)
    d[0, :wl.n_nodes] = torch.from_numpy(np.random.default_rng(8).normal(size=wl.n_nodes))
    d[1:, :wl.n_nodes] = 1e-3 * torch.from_numpy(np.random.default_rng(9).normal(size=(3, wl.n_nodes)))
    Lp = loss(run_gpu(s, wl, wl.sigma_field, wl.params, y0 + EPS * d, sens), target)
    Lm = loss(run_gpu(s, wl, wl.sigma_field, wl.params, y0 - EPS * d, sens), target)
    fd = (Lp - Lm) / (2 * EPS)
    ad = float((gy0 * d).sum())
    assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)


def run_oracle(wl, sig, params, sens):
    w = I.hh_field_sheet(16)
    w.sigma_field = sig
    w.params = params
    m = O.Monodomain(w, cg_tol=1e-15)
    y = m.init_state()
    out = []
    t = 0.0
    for _ in range(NSTEPS):
        y, _, _, _ = m.step(y, t, w.dt, w.M, w.K)
        t += w.dt
        out.append(y[0][sens])
    return np.array(out)


def test_adjoint_vs_oracle_finite_differences(case):
    """The oracle's forward map (independent of the CUDA path), differentiated by
    central differences, against the GPU adjoint."""
    wl, s, y0, sens, target = case
    tr, gsig, gpar, _ = gradients(case)
    tr_o = run_oracle(wl, wl.sigma_field, wl.params, sens)
    assert np.abs(tr - tr_o).max() < 1e-10 * np.abs(tr_o).max()
    d = wl.sigma_field * np.random.default_rng(4).normal(size=wl.n_nodes)
    fd = (loss(run_oracle(wl, wl.sigma_field + EPS * d, wl.params, sens), target)
          - loss(run_oracle(wl, wl.sigma_field - EPS * d, wl.params, sens), target)) / (2 * EPS)
    assert abs(float(gsig @ d) - fd) <= 1e-5 * abs(fd)
    p = wl.params.copy()
    h = EPS * p[0]
    pp, pm = p.copy(), p.copy()
    pp[0] += h
    pm[0] -= h
    fd = (loss(run_oracle(wl, wl.sigma_field, pp, sens), target)
          - loss(run_oracle(wl, wl.sigma_field, pm, sens), target)) / (2 * h)
    assert abs(gpar[0] - fd) <= 1e-5 * abs(fd)


def test_autograd_function_matches_adjoint(case):
    wl, s, y0, sens, target = case
    _, gsig, gpar, _ = gradients(case)
    sig = torch.from_numpy(wl.sigma_field.copy()).requires_grad_(True)
    gna = torch.tensor(float(wl.params[0]), dtype=torch.float64, requires_grad=True)
    gk = torch.tensor(float(wl.params[1]), dtype=torch.float64, requires_grad=True)
    tr = E.sensor_traces(s, sig, gna, gk, y0, 0.0, wl.dt, wl.M, wl.K, NSTEPS, torch.from_numpy(sens).cuda())
    L = 0.5 * ((tr - torch.from_numpy(target).cuda()) ** 2).sum()
    L.backward()
    np.testing.assert_allclose(sig.grad.numpy(), gsig, rtol=1e-12, atol=1e-18)
    assert abs(gna.grad.item() - gpar[0]) <= 1e-12 * abs(gpar[0])
    assert abs(gk.grad.item() - gpar[1]) <= 1e-12 * abs(gpar[1])


# ---------------------------------------------------------------- against the oracle's discrete adjoint

def _gpu_and_oracle_gradients(n, nsteps, nsens, seed):
    from oracle.adjoint import HHFieldAdjoint
    wl = I.hh_field_sheet(n)
    rng = np.random.default_rng(seed)
    sens = np.sort(rng.choice(wl.n_nodes, size=nsens, replace=False)).astype(np.int32)
    s = P.Solver.from_workload(wl, M_max=wl.M)
    y0 = s.new_state()
    s.init_state(y0, wl.V0)
    sd = torch.from_numpy(sens).cuda()

    def forward(sig, params, want_ckpt):
        s.set_params(params)
        s.set_conductivity_field(sig)
        y = y0.clone()
        tr = torch.empty((nsteps, nsens), dtype=torch.float64, device="cuda")
        ck = torch.empty((nsteps, s.n_state, s.ld), dtype=torch.float64, device="cuda")
        s.adjoint_forward(y, 0.0, wl.dt, wl.M, wl.K, nsteps, sd, tr, ck)
        assert s.residual()[0] == 0
        torch.cuda.synchronize()
        return tr.cpu().numpy(), ck

    p = wl.params.copy()
    p[0] *= 1.05
    p[1] *= 0.95
    target, _ = forward(I.lognormal_field(n, n, 1, seed=seed + 1), p, False)
    tr, ck = forward(wl.sigma_field, wl.params, True)
    dtr = tr - target
    gsig, gpar, gy0 = s.adjoint_backward(ck, 0.0, wl.dt, wl.M, wl.K, nsteps, sd, torch.from_numpy(dtr).cuda(),
                                         want_y0=True)
    torch.cuda.synchronize()
    gpu = (gsig.cpu().numpy(), float(gpar[0]), float(gpar[1]), gy0[:, :wl.n_nodes].cpu().numpy())
    adj = HHFieldAdjoint(O.Monodomain(wl, cg_tol=1e-15))
    y0c = y0[:, :wl.n_nodes].cpu().numpy()
    tr_o, _ = adj.traces(y0c, 0.0, wl.dt, wl.M, wl.K, nsteps, sens)
    assert np.abs(tr - tr_o).max() < 1e-10 * np.abs(tr_o).max()
    orc = adj.sensor_gradients(y0c, 0.0, wl.dt, wl.M, wl.K, nsteps, sens, dtr)
    return gpu, orc


def _compare(gpu, orc, tol):
    (gs, gna, gk, gy), (os_, ona, ok, oy) = gpu, orc
    assert np.abs(os_).max() > 0 and ona != 0 and ok != 0
    # the conductivity field, node by node (max-norm relative)
    assert np.abs(gs - os_).max() <= tol * np.abs(os_).max(), np.abs(gs - os_).max() / np.abs(os_).max()
    assert abs(gna - ona) <= tol * abs(ona), (gna, ona)
    assert abs(gk - ok) <= tol * abs(ok), (gk, ok)
    for s in range(oy.shape[0]):                 # every state of every node
        assert np.abs(gy[s] - oy[s]).max() <= tol * np.abs(oy[s]).max(), (s, np.abs(gy[s] - oy[s]).max())


def test_adjoint_matches_oracle_adjoint_16x16():
    """The GPU adjoint (esdc_adjoint_backward) against the oracle's discrete
    adjoint on the 16x16 field sheet over 30 steps: every component of
    dL/dsigma and dL/dy0, and dL/dg_Na, dL/dg_K, within 1e-9 (max-norm
    relative).  Both differentiate the same step map; their forward solves stop
    at relative residuals of 1e-14 (GPU) and 1e-15 (oracle)."""
    gpu, orc = _gpu_and_oracle_gradients(16, 30, 8, seed=41)
    _compare(gpu, orc, 1e-9)


@pytest.mark.slow
def test_adjoint_matches_oracle_adjoint_32x32_100_steps():
    gpu, orc = _gpu_and_oracle_gradients(32, 100, 16, seed=43)
    _compare(gpu, orc, 1e-9)
