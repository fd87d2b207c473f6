"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element
by element on seeded inputs.  Tolerances: the hot path is FP64 end to end, so
single kernels agree to a few ulps times the conditioning of the step (stated
per test); multi-step runs are held to the 1e-10 relative max-norm bound on V.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import oracle as O  # noqa: E402
import paper_2405_19994_gb300 as P  # noqa: E402
from paper_2405_19994_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    P.lib()


def to_dev(solver, y):
    t = solver.new_state()
    t[:, : y.shape[1]] = torch.from_numpy(np.ascontiguousarray(y))
    return t


def from_dev(solver, t):
    torch.cuda.synchronize()
    return t[:, : solver.n_nodes].cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---------------------------------------------------------------- coefficient kernel (App. A)

@pytest.mark.parametrize("M", range(1, 9))
def test_coefficients_match_oracle(M):
    wl = I.hh_sheet_32().with_mesh(4, 4, 1)
    s = P.Solver.from_workload(wl)
    zs = -np.concatenate([[0.0, 1e-14, 1e-9, 1e-5], np.linspace(1e-3, 12, 97), np.logspace(1, 3.5, 40)])
    a_gpu = s.coefficients(torch.from_numpy(zs).cuda(), M).cpu().numpy()
    w = np.abs(O.fornberg_weights(M)).max()
    for e, z in enumerate(zs):
        a_orc = O.aij(M, z)
        # rounding of sum_k c_i^k w_j^{k-1} phi_k grows with max|w| (both sides use the sum)
        np.testing.assert_allclose(a_gpu[:, :, e], a_orc, rtol=0, atol=16 * 2.2e-16 * max(1.0, w),
                                   err_msg=f"z={z}")


# ---------------------------------------------------------------- FP64 exp / reciprocal

def test_library_exp_and_reciprocal_error_bounds():
    from paper_2405_19994_gb300 import esdc as E
    rng = np.random.default_rng(0)
    x = np.concatenate([np.linspace(-706.9, 709.7, 200001), rng.uniform(-50, 50, 200000),
                        rng.uniform(-1e-3, 1e-3, 10000), [0.0, -0.0, 1e-300, -1e-300]])
    xd = torch.from_numpy(x).cuda()
    ex, _ = E.math_check(xd)
    ref = torch.exp(xd)                    # CUDA's exp
    ulp = torch.abs(ex - ref) / torch.abs(torch.nextafter(ref, torch.full_like(ref, np.inf)) - ref)
    assert float(ulp.max()) <= 2.0, float(ulp.max())
    # special values
    sp = torch.tensor([-800.0, 710.0, float("nan"), float("inf"), -float("inf")], dtype=torch.float64).cuda()
    e2, _ = E.math_check(sp)
    e2 = e2.cpu().numpy()
    assert e2[0] == 0.0 and np.isinf(e2[1]) and np.isnan(e2[2]) and np.isinf(e2[3]) and e2[4] == 0.0
    d = np.concatenate([np.geomspace(1e-30, 1e290, 100001), -np.geomspace(1e-30, 1e290, 1001),
                        1 + rng.uniform(0, 1e12, 100000),
                        # every region of the mantissa, at many binades and both signs
                        np.ldexp(1 + rng.uniform(0, 1, 1000000), rng.integers(-95, 95, 1000000))
                        * rng.choice([-1.0, 1.0], 1000000)])
    dd = torch.from_numpy(d).cuda()
    _, rc = E.math_check(dd)
    ref = 1.0 / dd
    ulp = torch.abs(rc - ref) / torch.abs(torch.nextafter(ref, torch.full_like(ref, np.inf)) - ref)
    assert float(ulp.max()) <= 2.0, float(ulp.max())


# ---------------------------------------------------------------- ionic models

@pytest.mark.parametrize("model", [I.MODEL_HH1952, I.MODEL_SYN19])
def test_ionic_pointwise(model):
    wl = I.hh_sheet_32() if model == I.MODEL_HH1952 else I.syn19_slab()
    wl = wl.with_mesh(37, 5, 1)
    s = P.Solver.from_workload(wl)
    y = I.random_state(wl, seed=11)
    y[0] = np.linspace(-110, 70, wl.n_nodes)
    y[0, 3] = wl.params[6] + 25.0 if model == I.MODEL_HH1952 else y[0, 3]    # alpha_m's 0/0 point
    y[0, 4] = wl.params[6] + 10.0 if model == I.MODEL_HH1952 else y[0, 4]    # alpha_n's 0/0 point
    fE, lam, yinf = (from_dev(s, t) for t in s.ionic(to_dev(s, y)))
    for p in range(wl.n_nodes):
        f0, l0, i0 = O.ionic_point(model, wl.params, y[:, p])
        np.testing.assert_allclose(fE[:, p], f0, rtol=4e-14, atol=1e-15)
        np.testing.assert_allclose(lam[:, p], l0, rtol=4e-14, atol=0)
        np.testing.assert_allclose(yinf[:, p], i0, rtol=4e-14, atol=1e-300)


@pytest.mark.parametrize("model", [I.MODEL_HH1952, I.MODEL_SYN19])
def test_gate_table_range_and_edges(model):
    """The gate functions come from the handle's V table on [-140, 100) mV and
    from the direct formulas outside it: both against the oracle from -300 to
    +200 mV, at the table's edges and at points 1e-9 mV either side of them,
    and a NaN potential stays NaN."""
    wl = I.hh_sheet_32() if model == I.MODEL_HH1952 else I.syn19_slab()
    edges = [-140.0, -140.0 + 1e-9, -140.0 - 1e-9, -139.5, -0.5, 0.0, 99.5, 100.0 - 1e-9, 100.0, 100.0 + 1e-9]
    V = np.concatenate([np.linspace(-300.0, 200.0, 1001), edges, [np.nan]])
    wl = wl.with_mesh(len(V), 1, 1)
    s = P.Solver.from_workload(wl)
    y = I.random_state(wl, seed=13)
    y[0] = V
    fE, lam, yinf = (from_dev(s, t) for t in s.ionic(to_dev(s, y)))
    for p in range(wl.n_nodes - 1):
        f0, l0, i0 = O.ionic_point(model, wl.params, y[:, p])
        np.testing.assert_allclose(lam[:, p], l0, rtol=4e-14, atol=0, err_msg=f"V={V[p]}")
        np.testing.assert_allclose(yinf[:, p], i0, rtol=4e-14, atol=1e-300, err_msg=f"V={V[p]}")
        np.testing.assert_allclose(fE[:, p], f0, rtol=4e-14, atol=1e-15, err_msg=f"V={V[p]}")
    gates = slice(1 + (0 if model == I.MODEL_HH1952 else 6), None)
    assert np.all(np.isnan(lam[gates, -1])) and np.all(np.isnan(yinf[gates, -1]))


@pytest.mark.parametrize("model", [I.MODEL_HH1952, I.MODEL_SYN19])
def test_init_state(model):
    wl = (I.hh_sheet_32() if model == I.MODEL_HH1952 else I.syn19_slab()).with_mesh(7, 3, 2)
    s = P.Solver.from_workload(wl)
    y = s.new_state()
    s.init_state(y, wl.V0)
    got = from_dev(s, y)
    want = O.Monodomain(wl).init_state()
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-300)


# ---------------------------------------------------------------- diffusion solve (CG) vs DCT-II

@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 1, 1), (33, 17, 1), (19, 13, 7), (64, 48, 5)])
@pytest.mark.parametrize("g", [1e-3, 0.05, 2.0])
def test_diffusion_solve_matches_dct(shape, g):
    # the iterative solves (solver "cheb": Chebyshev where the spectrum is
    # known, CG elsewhere) against the exact DCT-II
    nx, ny, nz = shape
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    s = P.Solver.from_workload(wl, cg_maxit=2000, solver="cheb")
    m = O.Monodomain(wl)
    rng = np.random.default_rng(5)
    b = rng.normal(size=wl.n_nodes)
    x0 = rng.normal(size=wl.n_nodes)
    want = m.solve_shifted(g, b, method=O.SOLVE_DCT)
    bd = torch.from_numpy(b).cuda()
    xd = torch.from_numpy(x0).cuda()
    it = s.diffusion_solve(g, bd, xd)
    got = xd.cpu().numpy()
    # ||x - x*|| <= kappa * tol * ||x*|| with kappa = 1 + 4 d g / h^2
    kappa = 1 + 4 * 3 * g / wl.h**2
    assert rel(got, want) < 50 * kappa * 1e-14, (rel(got, want), it)
    assert it <= 2000


# ---------------------------------------------------------------- Chebyshev semi-iteration

def _spectrum_hi(wl, g):
    return 1 + g / wl.h**2 * sum(4 * math.sin(math.pi * (n - 1) / (2 * n)) ** 2
                                 for n in (wl.nx, wl.ny, wl.nz) if n > 1)


@pytest.mark.parametrize("shape", [(4, 1, 1), (64, 1, 1), (32, 24, 1), (48, 40, 9), (8, 3, 17)])
@pytest.mark.parametrize("g", [1e-3, 0.05, 2.0])
def test_chebyshev_solve_matches_dct(shape, g):
    """solver="cheb" on scalar-sigma meshes with nx % 4 == 0 takes the
    Chebyshev semi-iteration; both solvers against the exact DCT-II solve."""
    nx, ny, nz = shape
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    m = O.Monodomain(wl)
    rng = np.random.default_rng(17)
    b = rng.normal(size=wl.n_nodes)
    x0 = rng.normal(size=wl.n_nodes)
    want = m.solve_shifted(g, b, method=O.SOLVE_DCT)
    tol = 1e-14
    kappa = _spectrum_hi(wl, g)
    its = {}
    for solver in ("cheb", "cg"):
        s = P.Solver.from_workload(wl, cg_maxit=4000, tol_cg=tol, solver=solver)
        xd = torch.from_numpy(x0).cuda()
        its[solver] = s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
        got = xd.cpu().numpy()
        assert rel(got, want) < 50 * kappa * tol, (solver, rel(got, want), its[solver])
    # The Chebyshev run stops at the first k with 2 q^k ||r_0|| <= tol ||b||,
    # q = (sqrt(kappa) - 1)/(sqrt(kappa) + 1), then checks every two iterations
    # if rounding left the residual short; a CG run would not follow this count.
    r0 = b - (x0 - g * m.laplacian(x0))
    q = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    k = max(1, math.ceil(math.log(0.5 * tol * np.linalg.norm(b) / np.linalg.norm(r0)) / math.log(q)))
    assert k - 1 <= its["cheb"] <= k + 6, (its, k)


def test_chebyshev_zero_shift_and_ineligible_meshes():
    # g = 0 is the identity, and a g whose interval 1 + g w/h^2 rounds to 1 has
    # no width either (the CG runs); nx not a multiple of 4 takes the
    # one-node-per-thread Chebyshev kernel; all give the exact result.
    rng = np.random.default_rng(4)
    for shape, g in (((16, 8, 1), 0.0), ((16, 8, 1), 1e-19), ((18, 7, 3), 0.3)):
        wl = I.hh_sheet_32().with_mesh(*shape)
        m = O.Monodomain(wl)
        b = rng.normal(size=wl.n_nodes)
        s = P.Solver.from_workload(wl, cg_maxit=2000, solver="cheb")
        xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
        s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
        want = m.solve_shifted(g, b, method=O.SOLVE_DCT)
        assert rel(xd.cpu().numpy(), want) < 50 * _spectrum_hi(wl, g) * 1e-14


@pytest.mark.parametrize("solver", ["auto", "cheb", "cg"])
def test_one_step_either_solver_matches_oracle(solver):
    wl = I.syn19_slab().with_mesh(16, 12, 5)
    M, K = 4, 6
    s = P.Solver.from_workload(wl, M_max=M, solver=solver)
    y0 = I.random_state(wl, seed=31)
    yd = to_dev(s, y0)
    s.sweep(yd, 0.5, wl.dt, M, K)
    assert s.residual()[0] == 0
    got = from_dev(s, yd)
    want, _, _, _ = O.Monodomain(wl).step(y0, 0.5, wl.dt, M, K)
    for srow in range(wl.n_state):
        scale = max(np.abs(want[srow]).max(), 1e-3)
        assert np.abs(got[srow] - want[srow]).max() / scale < 1e-12, (solver, srow)


# ---------------------------------------------------------------- DCT-II direct solve (options.solver = 2)

@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 1, 1), (33, 17, 1), (19, 13, 7), (64, 48, 5), (2, 3, 2),
                                   (128, 8, 4), (8, 128, 3), (16, 16, 16), (256, 3, 2), (2, 2, 64), (32, 1, 1),
                                   # the fused y-z kernel (second order, ny a power of two >= 16, nz >= 2):
                                   # odd nz, nx = 1, and more than a warp per line pair (ny 256, 512)
                                   (4, 32, 7), (1, 16, 4), (1, 64, 9), (3, 256, 3), (5, 512, 2)])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("g", [1e-3, 0.05, 2.0])
def test_dct_solve_matches_oracle(shape, order, g):
    """The GPU DCT-II solve (FFT of line pairs along power-of-two axes, dense
    products along the others, tridiagonal z solve for the second order)
    against the oracle's exact DCT-II solve of the same stencil."""
    nx, ny, nz = shape
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.order = order
    s = P.Solver.from_workload(wl, solver="dct")
    m = O.Monodomain(wl)
    rng = np.random.default_rng(23)
    b = rng.normal(size=wl.n_nodes)
    want = m.solve_shifted(g, b, method=O.SOLVE_DCT)
    xd = torch.from_numpy(rng.normal(size=wl.n_nodes)).cuda()     # the initial guess plays no part
    it = s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
    got = xd.cpu().numpy()
    assert it == 1
    # both are exact solves; the oracle's transform is a plain O(n^2) sum whose
    # rounding grows with the axis length (about 2e-14 at n = 256)
    assert rel(got, want) < 1e-13, rel(got, want)
    # and the residual of the oracle's own operator is at rounding level
    Bx = got - g * m.laplacian(got)
    assert np.abs(Bx - b).max() < 1e-12 * (1 + 16 * 3 * g / wl.h**2) * np.abs(b).max()


@pytest.mark.slow
@pytest.mark.parametrize("g", [0.05 * 0.1214 * 0.0885, 0.05 * 0.1214 * 0.4])
def test_dct_solve_full_slab(g):
    """The DCT solve on the full 128x128x32 slab of the headline workload (the
    FFT path along x and y with the launch shape the bench uses, the
    tridiagonal z solve), for two of its implicit rows' g, against the oracle's
    CG solved to 1e-15 (its O(n^2) DCT sums are less accurate than the solve
    under test at n = 128)."""
    wl = I.syn19_slab()
    s = P.Solver.from_workload(wl, solver="dct")
    m = O.Monodomain(wl, solver=O.SOLVE_CG, cg_tol=1e-15, cg_maxit=500)
    rng = np.random.default_rng(29)
    b = rng.normal(size=wl.n_nodes)
    want = m.solve_shifted(g, b, method=O.SOLVE_CG)
    xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
    for _ in range(2):                    # the second call reuses the cached z-factors of g
        assert s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd) == 1
        got = xd.cpu().numpy()
        assert rel(got, want) < 1e-13, rel(got, want)
    Bx = got - g * m.laplacian(got)
    assert np.abs(Bx - b).max() < 1e-14 * np.abs(b).max() * (1 + 12 * g / wl.h**2)


@pytest.mark.parametrize("order", [2, 4])
def test_dct_one_step_matches_oracle(order):
    wl = I.syn19_slab().with_mesh(12, 10, 4)
    wl.order = order
    M, K = 4, 6
    s = P.Solver.from_workload(wl, M_max=M, solver="dct")
    y0 = I.random_state(wl, seed=41)
    yd = to_dev(s, y0)
    s.sweep(yd, 0.5, wl.dt, M, K)
    assert s.residual()[0] == 0
    assert (s.stats(K * M) == 1).all()
    got = from_dev(s, yd)
    want, _, _, _ = O.Monodomain(wl).step(y0, 0.5, wl.dt, M, K)
    for srow in range(wl.n_state):
        scale = max(np.abs(want[srow]).max(), 1e-3)
        assert np.abs(got[srow] - want[srow]).max() / scale < 1e-12, (order, srow)


def test_dct_needs_scalar_sigma():
    wl = I.hh_sheet_32().with_mesh(16, 12, 1)
    s = P.Solver.from_workload(wl, solver="dct")
    with pytest.raises(P.EsdcError) as e:
        s.set_conductivity_field(I.lognormal_field(wl.nx, wl.ny, wl.nz, seed=3))
    assert e.value.code == -6
    with pytest.raises(P.EsdcError) as e:
        s.set_conductivity_layers(I.fibre_layers(1))
    assert e.value.code == -6


# ---------------------------------------------------------------- one HSDC step

CASES = [
    # (model, mesh, M, K, t0)
    (I.MODEL_HH1952, (12, 10, 1), 3, 4, 0.5),
    (I.MODEL_HH1952, (9, 7, 3), 2, 3, 0.2),
    (I.MODEL_HH1952, (33, 1, 1), 1, 2, 0.0),
    (I.MODEL_HH1952, (6, 5, 1), 8, 3, 1.7),
    (I.MODEL_HH1952, (1, 1, 1), 3, 4, 0.0),
    (I.MODEL_HH1952, (10, 9, 1), 3, 0, 0.5),
    (I.MODEL_SYN19, (11, 6, 4), 4, 6, 0.5),
    (I.MODEL_SYN19, (40, 3, 1), 3, 2, 0.9),
    (I.MODEL_SYN19, (7, 7, 2), 6, 5, 0.0),
]


@pytest.mark.parametrize("model,mesh,M,K,t0", CASES)
def test_one_step_matches_oracle(model, mesh, M, K, t0):
    base = I.hh_sheet_32() if model == I.MODEL_HH1952 else I.syn19_slab()
    wl = base.with_mesh(*mesh)
    wl.boxes = np.array([[0, 2, 0, 3, 0, 2]], np.int32)       # stimulus on a corner box, on for t < 1
    dt = wl.dt
    s = P.Solver.from_workload(wl, M_max=M)
    s.keep_residual(True)
    y0 = I.random_state(wl, seed=hash((model, mesh, M, K)) % 1000)
    yd = to_dev(s, y0)
    s.sweep(yd, t0, dt, M, K)
    rc, res_inf, y_inf, res_state = s.residual()
    col, res = s.collocation(M, with_residual=True)
    got = from_dev(s, yd)
    col = col[:, :, : wl.n_nodes].cpu().numpy()
    res = res[:, :, : wl.n_nodes].cpu().numpy()
    m = O.Monodomain(wl, solver=O.SOLVE_DCT)
    want, st, wcol, wres = m.step(y0, t0, dt, M, K, want_colloc=True, want_resid=True)
    assert rc == 0
    # per state: relative to that state's scale
    for srow in range(wl.n_state):
        scale = max(np.abs(want[srow]).max(), 1e-3)
        assert np.abs(got[srow] - want[srow]).max() / scale < 1e-12, (srow, np.abs(got[srow] - want[srow]).max())
        for i in range(M):
            assert np.abs(col[i, srow] - wcol[i, srow]).max() / scale < 1e-12
    # residual vectors: absolute, scaled by dt*|G| (the residual is a difference of O(1) terms)
    rscale = max(np.abs(wres).max(), 1e-12 * y_inf)
    assert np.abs(res - wres).max() <= 1e-12 * max(y_inf, 1.0) + 1e-9 * rscale
    assert math.isclose(res_inf, np.abs(res).max(), rel_tol=0, abs_tol=0)
    assert y_inf == max(np.abs(y0).max(), np.abs(col).max())



@pytest.mark.parametrize("model,mesh,M,K,precision,solver", [
    (I.MODEL_HH1952, (32, 32, 1), 3, 4, "fp64", "auto"),
    (I.MODEL_HH1952, (21, 9, 3), 2, 1, "fp64", "cheb"),
    (I.MODEL_HH1952, (16, 16, 4), 4, 2, "mixed", "auto"),
    (I.MODEL_HH1952, (12, 8, 1), 1, 3, "fp64", "auto"),       # M = 1: never fused
    (I.MODEL_HH1952, (12, 8, 1), 3, 0, "fp64", "auto"),       # K = 0: no sweep
    (I.MODEL_SYN19, (16, 16, 8), 4, 6, "fp64", "auto"),
    (I.MODEL_SYN19, (11, 6, 4), 5, 3, "fp64", "cg"),
])
def test_fused_node1_equals_separate_launches(model, mesh, M, K, precision, solver):
    # Node 1 of each sweep inside the set-up / previous final-evaluation launch
    # (the default) against its own launch: the same state, iterate, residual
    # vectors and residual norms, bit for bit, over three steps.
    base = I.hh_sheet_32() if model == I.MODEL_HH1952 else I.syn19_slab()
    wl = base.with_mesh(*mesh)
    wl.boxes = np.array([[0, 3, 0, 3, 0, 2]], np.int32)
    y0 = I.random_state(wl, seed=7)
    out = []
    for fuse in (True, False):
        s = P.Solver.from_workload(wl, M_max=M, precision=precision, solver=solver, fuse_node1=fuse)
        s.keep_residual(True)
        if M >= 2:
            yd = to_dev(s, y0)
        else:                     # M = 1 diverges from a random state (the oracle too): start at rest
            yd = s.new_state()
            s.init_state(yd, wl.V0)
        t = 0.2
        for _ in range(3):
            s.sweep(yd, t, wl.dt, M, K)
            t += wl.dt
        rc, res_inf, y_inf, res_state = s.residual()
        col, res = s.collocation(M, with_residual=True)
        n = wl.n_nodes
        out.append((from_dev(s, yd), col[:, :, :n].cpu().numpy(), res[:, :, :n].cpu().numpy(), rc, res_inf, y_inf,
                    s.stats(max(M * K, 1))))
    (ya, ca, ra, rca, ria, yia, ita), (yb, cb, rb, rcb, rib, yib, itb) = out
    assert rca == rcb == 0
    np.testing.assert_array_equal(ya, yb)
    np.testing.assert_array_equal(ca, cb)
    np.testing.assert_array_equal(ra, rb)
    assert (ria, yia) == (rib, yib)
    np.testing.assert_array_equal(ita, itb)


@pytest.mark.parametrize("dt", [1.0, 0.05])
def test_setup_table_and_direct_coefficients_match_oracle(dt):
    # The set-up takes dt S_ij and dt d_i phi_1 from a table in z = dt Lambda
    # for |z| < 4095 and evaluates them directly beyond.  With dt = 1 ms the
    # synthetic model's fastest gates (Lambda down to -5189/ms) fall beyond the
    # table, so one node mixes both.  The same step twice from the same state.
    wl = I.syn19_slab().with_mesh(9, 7, 3)
    y0 = I.random_state(wl, seed=11)
    s = P.Solver.from_workload(wl, M_max=3)
    want = O.Monodomain(wl, solver=O.SOLVE_DCT).step(y0, 0.0, dt, 3, 2)[0]
    for _ in range(2):
        yd = to_dev(s, y0)
        s.sweep(yd, 0.0, dt, 3, 2)
        assert s.residual()[0] == 0
        got = from_dev(s, yd)
        for srow in range(wl.n_state):
            scale = max(np.abs(want[srow]).max(), 1e-3)
            assert np.abs(got[srow] - want[srow]).max() / scale < 1e-11, (srow, np.abs(got[srow] - want[srow]).max())


def test_setup_tables_for_many_step_sizes():
    # A handle keeps four set-up coefficient tables (one per (M, dt)); a fifth
    # step size replaces the oldest.  Every step matches the oracle, and a step
    # size whose table was replaced gives the bits it gave before once its
    # table is rebuilt.
    wl = I.hh_sheet_32().with_mesh(12, 9, 2)
    y0 = I.random_state(wl, seed=5)
    s = P.Solver.from_workload(wl, M_max=3)
    m = O.Monodomain(wl, solver=O.SOLVE_DCT)
    first = None
    for dt in [0.025, 0.01, 0.02, 0.03, 0.04, 0.05, 0.025]:
        want = m.step(y0, 0.2, dt, 3, 2)[0]
        for _ in range(2):
            yd = to_dev(s, y0)
            s.sweep(yd, 0.2, dt, 3, 2)
            assert s.residual()[0] == 0
            got = from_dev(s, yd)
            for srow in range(wl.n_state):
                scale = max(np.abs(want[srow]).max(), 1e-3)
                assert np.abs(got[srow] - want[srow]).max() / scale < 1e-12, (dt, srow)
        if first is None:
            first = got
    np.testing.assert_array_equal(got, first)


@pytest.mark.parametrize("nx,solver", [(16, "cheb"), (15, "cheb"), (16, "cg"), (15, "cg")])
def test_errors_reported(nx, solver):
    # nx = 16 takes the quad-form kernels, nx = 15 the one-node-per-thread ones
    wl = I.hh_sheet_32().with_mesh(nx, 16, 1)
    s = P.Solver.from_workload(wl, M_max=3, cg_maxit=1, tol_cg=1e-15, solver=solver)
    y = to_dev(s, I.random_state(wl, seed=1))
    with pytest.raises(P.EsdcError) as e:
        s.sweep(y, 0.0, wl.dt, 4, 2)                          # M > M_max
    assert e.value.code == -1
    s.sweep(y, 0.0, wl.dt, 3, 2)
    rc, *_ = s.residual()
    assert rc == -3                                           # CG_NOT_CONVERGED
    s2 = P.Solver.from_workload(wl, M_max=3, solver=solver)
    y2 = I.random_state(wl, seed=2)
    y2[0, 17] = np.nan
    yd = to_dev(s2, y2)
    s2.sweep(yd, 0.0, wl.dt, 3, 2)
    rc, *_ = s2.residual()
    assert rc == -4                                           # NONFINITE
    s3 = P.Solver.from_workload(wl, M_max=3, solver=solver)
    yd = to_dev(s3, I.random_state(wl, seed=2))
    s3.sweep(yd, 0.0, wl.dt, 3, 2)
    assert s3.residual()[0] == 0                              # a fresh handle is clean
    it = s3.stats(6)
    assert np.all(it >= 1) and np.all(it < 200)


def test_dct_errors_reported():
    # the automatic solver on the scalar sigma is the direct DCT solve: no
    # iteration limit applies (every solve reports one "iteration"), and a NaN
    # in the state still raises NONFINITE
    wl = I.hh_sheet_32().with_mesh(16, 16, 1)
    s = P.Solver.from_workload(wl, M_max=3, cg_maxit=1, tol_cg=1e-15)
    y = to_dev(s, I.random_state(wl, seed=1))
    s.sweep(y, 0.0, wl.dt, 3, 2)
    assert s.residual()[0] == 0
    assert (s.stats(6) == 1).all()
    y2 = I.random_state(wl, seed=2)
    y2[0, 17] = np.nan
    yd = to_dev(s, y2)
    s.sweep(yd, 0.0, wl.dt, 3, 2)
    assert s.residual()[0] == -4                              # NONFINITE



def _solve_matches_oracle(s, wl, seed=3):
    m = O.Monodomain(wl)
    b = np.random.default_rng(seed).normal(size=wl.n_nodes)
    g = 0.3 * 0.17
    xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
    s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
    return rel(xd.cpu().numpy(), m.solve_shifted(g, b))


def test_auto_solver_takes_the_dct_only_where_it_is_cheap():
    # "auto" on the FP64 path with the scalar sigma: the DCT-II where every
    # transformed axis is of power-of-two length or the dense ones add up to
    # at most 32; the Chebyshev semi-iteration otherwise (a dense axis costs
    # n FMAs per value and pass)
    base = I.hh_sheet_32()
    for shape, want in [((32, 32, 1), "dct"), ((32, 24, 1), "dct"), ((13, 11, 1), "dct"),
                        ((48, 40, 1), "cheb"), ((64, 33, 1), "cheb"), ((16, 16, 40), "dct")]:
        wl = base.with_mesh(*shape)
        s = P.Solver.from_workload(wl)
        assert s.solver_in_use() == want, shape
        assert _solve_matches_oracle(s, wl) < 1e-12, shape
    # the fourth order transforms z as well: nz = 40 is a dense axis of 40
    wl = base.with_mesh(16, 16, 40)
    s = P.Solver.from_workload(wl)
    s.set_stencil_order(4)
    assert s.solver_in_use() == "cheb"
    wl4 = base.with_mesh(16, 16, 40)
    wl4.order = 4
    assert _solve_matches_oracle(s, wl4) < 1e-12
    s.set_stencil_order(2)
    assert s.solver_in_use() == "dct"
    # a conductivity field is not diagonalised by the DCT
    sig = np.random.default_rng(4).uniform(0.05, 0.2, size=wl.n_nodes)
    s.set_conductivity_field(sig)
    assert s.solver_in_use() == "cheb"
    s.set_conductivity_field(None)
    assert s.solver_in_use() == "dct"
    # explicit choices and the precision form
    assert P.Solver.from_workload(wl, solver="cg").solver_in_use() == "cg"
    assert P.Solver.from_workload(wl, solver="cheb").solver_in_use() == "cheb"
    assert P.Solver.from_workload(wl, solver="dct").solver_in_use() == "dct"
    assert P.Solver.from_workload(wl, precision="mixed").solver_in_use() == "cheb"


# ---------------------------------------------------------------- precision form (FP32 ionic model)

@pytest.mark.parametrize("shape", [(1, 1, 1), (37, 1, 1), (33, 17, 1), (19, 13, 7), (64, 48, 5), (16, 12, 3)])
@pytest.mark.parametrize("g", [1e-3, 0.05, 2.0])
@pytest.mark.parametrize("solver", ["auto", "cg"])
def test_refinement_solve_matches_dct(shape, g, solver):
    """Precision-form solve (FP32 inner solves, FP64 residuals): reaches the same
    FP64 tolerance as the FP64 CG, so it meets the same bound against the DCT.
    With solver "auto" and nx % 4 == 0 the inner solves are Chebyshev iterations."""
    nx, ny, nz = shape
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    s = P.Solver.from_workload(wl, cg_maxit=2000, precision="mixed", solver=solver)
    m = O.Monodomain(wl)
    rng = np.random.default_rng(6)
    b = rng.normal(size=wl.n_nodes)
    x0 = rng.normal(size=wl.n_nodes)
    want = m.solve_shifted(g, b, method=O.SOLVE_DCT)
    xd = torch.from_numpy(x0).cuda()
    s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
    kappa = 1 + 4 * 3 * g / wl.h**2
    assert rel(xd.cpu().numpy(), want) < 50 * kappa * 1e-14

@pytest.mark.parametrize("model,mesh,M,K", [(I.MODEL_HH1952, (12, 10, 1), 3, 4), (I.MODEL_SYN19, (11, 6, 4), 4, 6)])
def test_precision_form_one_step(model, mesh, M, K):
    """The precision form evaluates f_E, Lambda and y_inf in FP32; everything else
    is FP64.  One step from a seeded state: per state, the difference from the FP64
    oracle is bounded by the FP32 rounding of the ionic terms (relative 2^-23 ~ 1.2e-7)
    times the step's sensitivity: 1e-5 of the state's scale for V, 1e-5 absolute for
    the auxiliaries and gates."""
    base = I.hh_sheet_32() if model == I.MODEL_HH1952 else I.syn19_slab()
    wl = base.with_mesh(*mesh)
    s = P.Solver.from_workload(wl, M_max=M, precision="mixed")
    y0 = I.random_state(wl, seed=77)
    yd = to_dev(s, y0)
    s.sweep(yd, 0.4, wl.dt, M, K)
    assert s.residual()[0] == 0
    got = from_dev(s, yd)
    want, _, _, _ = O.Monodomain(wl).step(y0, 0.4, wl.dt, M, K)
    assert np.abs(got[0] - want[0]).max() <= 1e-5 * np.abs(want[0]).max()
    assert np.abs(got[1:] - want[1:]).max() <= 1e-5
    assert np.abs(got - want).max() > 0.0        # it really is a different (FP32) evaluation


def test_precision_form_hh_sheet_run():
    """32x32 HH sheet for 4 ms (160 steps) in the precision form against the oracle:
    the V error stays at the FP32 level (< 1e-4 relative in the max norm)."""
    wl = I.hh_sheet_32()
    s = P.Solver.from_workload(wl, precision="mixed")
    y = s.new_state()
    s.init_state(y, wl.V0)
    m = O.Monodomain(wl)
    ref = m.init_state()
    for n in range(wl.n_steps):
        s.sweep(y, n * wl.dt, wl.dt, wl.M, wl.K)
        ref, _, _, _ = m.step(ref, n * wl.dt, wl.dt, wl.M, wl.K)
    got = from_dev(s, y)
    err = rel(got[0], ref[0])
    assert err < 1e-4, err


# ---------------------------------------------------------------- layered anisotropic conductivity

@pytest.mark.parametrize("precision,solver", [("fp64", "auto"), ("fp64", "cheb"), ("fp64", "cg"), ("mixed", "auto")])
@pytest.mark.parametrize("shape", [(13, 11, 5), (40, 33, 3), (9, 9, 1), (16, 12, 6)])
def test_layered_solve_matches_oracle(precision, solver, shape):
    # fp64 with solver "auto" or "cheb" and nx % 4 == 0: the Chebyshev
    # semi-iteration on the Gershgorin interval of the layered operator
    nx, ny, nz = shape
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.layers = I.fibre_layers(nz)
    s = P.Solver.from_workload(wl, cg_maxit=2000, precision=precision, solver=solver)
    m = O.Monodomain(wl, solver=O.SOLVE_CG, cg_tol=1e-15)
    rng = np.random.default_rng(8)
    b = rng.normal(size=wl.n_nodes)
    g = 0.4
    want = m.solve_A(g, b)
    xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
    s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
    assert rel(xd.cpu().numpy(), want) < 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_layered_one_step_matches_oracle(precision, tol):
    """HH on a 3D slab with fibres rotating through the depth (the precision-form
    workload's physics, reduced mesh), one step from a mid-upstroke state.

    The start state comes from the oracle (rest, then 24 stimulated steps), not
    from random gates: HH with arbitrary gate values is far stiffer than any
    physical state, and at dt = 0.05 ms the sweep diverges from it on both sides."""
    wl = I.hh_aniso_slab().with_mesh(14, 12, 6)
    m = O.Monodomain(wl, cg_tol=1e-15)
    y0, t0 = m.init_state(), 0.0
    for _ in range(24):
        y0, _, _, _ = m.step(y0, t0, wl.dt, wl.M, wl.K)
        t0 += wl.dt
    assert y0[0].max() > 0.0 and y0[0].min() < -60.0              # a front is on the mesh
    s = P.Solver.from_workload(wl, M_max=wl.M, precision=precision)
    yd = to_dev(s, y0)
    s.sweep(yd, t0, wl.dt, wl.M, wl.K)
    assert s.residual()[0] == 0
    got = from_dev(s, yd)
    want, _, _, _ = m.step(y0, t0, wl.dt, wl.M, wl.K)
    assert np.abs(got[0] - want[0]).max() <= tol * np.abs(want[0]).max()
    assert np.abs(got[1:] - want[1:]).max() <= tol


@pytest.fixture(scope="module")
def aniso_full_step():
    """The oracle's step of the full precision-form workload (256x256x64, 4.2M
    nodes) from rest at t = 0, with the planar stimulus on (computed once)."""
    wl = I.hh_aniso_slab()
    m = O.Monodomain(wl, cg_tol=1e-15)
    y0 = m.init_state()
    want, _, _, _ = m.step(y0, 0.0, wl.dt, wl.M, wl.K)
    return wl, y0, want


@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_precision_workload_full_size_one_step(aniso_full_step, precision, tol):
    """The precision-form workload at full size in the configuration the bench
    times (default solver: the layered Chebyshev solve, or the Chebyshev
    refinement), one step, every element against the oracle."""
    wl, y0, want = aniso_full_step
    s = P.Solver.from_workload(wl, M_max=wl.M, precision=precision)
    yd = to_dev(s, y0)
    s.sweep(yd, 0.0, wl.dt, wl.M, wl.K)
    assert s.residual()[0] == 0
    got = from_dev(s, yd)
    assert np.abs(got[0] - want[0]).max() <= tol * np.abs(want[0]).max()
    assert np.abs(got[1:] - want[1:]).max() <= tol
    s.close()


@pytest.mark.slow
def test_field_sheet_full_size_steps():
    """The differentiation form's tissue at full size (256x256, log-normal field,
    the default solver: the field Chebyshev solve), 4 steps from rest with the
    corner stimulus on, every element against the oracle."""
    wl = I.hh_field_sheet()
    m = O.Monodomain(wl, cg_tol=1e-15)
    y = m.init_state()
    s = P.Solver.from_workload(wl, M_max=wl.M)
    yd = to_dev(s, y)
    t = 0.0
    for _ in range(4):
        s.sweep(yd, t, wl.dt, wl.M, wl.K)
        y, _, _, _ = m.step(y, t, wl.dt, wl.M, wl.K)
        t += wl.dt
    assert s.residual()[0] == 0
    got = from_dev(s, yd)
    assert np.abs(got[0] - y[0]).max() <= 1e-11 * np.abs(y[0]).max()
    assert np.abs(got[1:] - y[1:]).max() <= 1e-11


# ---------------------------------------------------------------- full workloads

def test_hh_sheet_full_run_matches_oracle():
    """32x32 HH sheet, corner stimulus, M=3, K=4, dt=0.025, T=4 ms (160 steps)."""
    wl = I.hh_sheet_32()
    s = P.Solver.from_workload(wl)
    y = s.new_state()
    s.init_state(y, wl.V0)
    m = O.Monodomain(wl)
    ref = m.init_state()
    np.testing.assert_allclose(from_dev(s, y), ref, rtol=1e-14)
    for n in range(wl.n_steps):
        s.sweep(y, n * wl.dt, wl.dt, wl.M, wl.K)
        ref, _, _, _ = m.step(ref, n * wl.dt, wl.dt, wl.M, wl.K)
        if n % 40 == 39:
            assert s.residual()[0] == 0
    got = from_dev(s, y)
    err = rel(got[0], ref[0])
    assert ref[0].max() > -60.0            # the wave is present in the sheet at T
    assert err < 1e-10, err
    assert got[1:].min() >= -1e-12 and got[1:].max() <= 1 + 1e-12


@pytest.mark.slow
def test_syn19_slab_full_size_one_step():
    """128x128x32 synthetic slab (524,288 nodes), M=4, K=6, dt=0.05: one step from a
    seeded mid-wave state, every output element against the oracle."""
    wl = I.syn19_slab()
    s = P.Solver.from_workload(wl, M_max=wl.M)
    y0 = I.random_state(wl, seed=2024)
    yd = to_dev(s, y0)
    s.sweep(yd, 0.5, wl.dt, wl.M, wl.K)
    rc, res_inf, y_inf, _ = s.residual()
    got = from_dev(s, yd)
    m = O.Monodomain(wl)
    want, st, _, _ = m.step(y0, 0.5, wl.dt, wl.M, wl.K)
    assert rc == 0
    for srow in range(wl.n_state):
        scale = max(np.abs(want[srow]).max(), 1e-3)
        assert np.abs(got[srow] - want[srow]).max() / scale < 1e-11, srow
    assert abs(res_inf - st["res_inf"]) <= 1e-9 * max(st["res_inf"], 1e-6)


# ---------------------------------------------------------------- heterogeneous conductivity field

@pytest.mark.parametrize("shape", [(13, 11, 1), (32, 24, 1), (9, 8, 5)])
@pytest.mark.parametrize("solver", ["auto", "cheb", "cg"])
def test_field_solve_matches_oracle(shape, solver):
    # "auto" and "cheb": the Chebyshev semi-iteration on the Gershgorin interval
    # of the field operator (the DCT does not diagonalise it)
    nx, ny, nz = shape
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.sigma_field = I.lognormal_field(nx, ny, nz, seed=7, corr=3.0)
    s = P.Solver.from_workload(wl, cg_maxit=2000, solver=solver)
    m = O.Monodomain(wl, solver=O.SOLVE_CG, cg_tol=1e-15)
    b = np.random.default_rng(9).normal(size=wl.n_nodes)
    g = 0.3
    want = m.solve_A(g, b)
    xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
    s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
    assert rel(xd.cpu().numpy(), want) < 1e-12


def test_field_run_matches_oracle():
    """HH on a 2D sheet with a log-normal conductivity field, corner stimulus:
    40 steps from rest against the oracle (the differentiation-form physics on a
    reduced mesh)."""
    wl = I.hh_field_sheet(32)
    s = P.Solver.from_workload(wl)
    y = s.new_state()
    s.init_state(y, wl.V0)
    m = O.Monodomain(wl, cg_tol=1e-15)
    ref = m.init_state()
    t = 0.0
    for _ in range(40):
        s.sweep(y, t, wl.dt, wl.M, wl.K)
        ref, _, _, _ = m.step(ref, t, wl.dt, wl.M, wl.K)
        t += wl.dt
    assert s.residual()[0] == 0
    got = from_dev(s, y)
    assert rel(got[0], ref[0]) < 1e-10
    assert np.abs(got[0]).max() > 0.0 and ref[0].max() > -60.0       # the corner has fired


def test_field_rejected_in_precision_form():
    wl = I.hh_sheet_32().with_mesh(8, 8, 1)
    s = P.Solver.from_workload(wl, precision="mixed")
    with pytest.raises(P.EsdcError) as e:
        s.set_conductivity_field(np.full(64, 0.2))
    assert e.value.code == -6


# ---------------------------------------------------------------- fourth-order Laplacian

@pytest.mark.parametrize("shape", [(13, 11, 1), (32, 24, 1), (9, 8, 5), (2, 3, 2)])
@pytest.mark.parametrize("solver", ["auto", "cheb", "cg"])
def test_order4_solve_matches_oracle(shape, solver):
    # "auto": the DCT-II solve; "cheb": the Chebyshev semi-iteration on the
    # exact fourth-order spectrum
    nx, ny, nz = shape
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.order = 4
    s = P.Solver.from_workload(wl, cg_maxit=2000, solver=solver)
    m = O.Monodomain(wl)                                   # the exact DCT-II solve
    b = np.random.default_rng(12).normal(size=wl.n_nodes)
    g = 0.3 * 0.17
    want = m.solve_shifted(g, b)
    xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
    s.diffusion_solve(g, torch.from_numpy(b).cuda(), xd)
    assert rel(xd.cpu().numpy(), want) < 1e-12


def test_order4_run_matches_oracle():
    """The parity sheet (32x32 HH, corner stimulus, M=3, K=4) with the paper's
    fourth-order differences: 60 steps against the oracle."""
    wl = I.hh_sheet_32()
    wl.order = 4
    s = P.Solver.from_workload(wl)
    y = s.new_state()
    s.init_state(y, wl.V0)
    m = O.Monodomain(wl)
    ref = m.init_state()
    t = 0.0
    for _ in range(60):
        s.sweep(y, t, wl.dt, wl.M, wl.K)
        ref, _, _, _ = m.step(ref, t, wl.dt, wl.M, wl.K)
        t += wl.dt
    assert s.residual()[0] == 0
    got = from_dev(s, y)
    assert rel(got[0], ref[0]) < 1e-10
    assert ref[0].max() > -60.0                            # the corner has fired


def test_order4_combinations_rejected():
    wl = I.hh_sheet_32().with_mesh(8, 8, 2)
    s = P.Solver.from_workload(wl)
    s.set_conductivity_layers(I.fibre_layers(2))
    with pytest.raises(P.EsdcError) as e:
        s.set_stencil_order(4)
    assert e.value.code == -6
    s2 = P.Solver.from_workload(wl, precision="mixed")
    with pytest.raises(P.EsdcError) as e:
        s2.set_stencil_order(4)
    assert e.value.code == -6
    s3 = P.Solver.from_workload(wl)
    s3.set_stencil_order(4)
    with pytest.raises(P.EsdcError) as e:
        s3.set_conductivity_field(np.full(wl.n_nodes, 0.2))
    assert e.value.code == -6


def test_fma_probe_counts_and_rates():
    from paper_2405_19994_gb300 import esdc as E
    ms64, fl64 = E.fma_probe(False, 2000)
    ms32, fl32 = E.fma_probe(True, 2000)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert fl64 == fl32 == 2 * 8 * 2000 * sms * 4 * 256
    assert ms64 > 0 and ms32 > 0
    assert fl32 / ms32 > 8 * fl64 / ms64          # FP32 issues many times faster than FP64 on this part
