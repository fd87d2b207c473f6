"""Failure detection on the GPU without a fault or a hang: the grid barrier of
the cooperative solve kernels gives up a wait after a bounded time and reports
ESDC_ERR_DEVICE_TIMEOUT, and the handle stays usable.  esdc_debug_barrier makes
the wait run out on purpose: one block does not arrive at the first barrier,
and every wait is limited to 2 ms (the arrival nobody makes is the flag nothing
sets).  Every wait in the library is bounded, so the test can only make the
kernel return early."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
import paper_2405_19994_gb300 as P  # noqa: E402
from paper_2405_19994_gb300 import inputs as I  # noqa: E402

TIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    P.lib()


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


# quad Chebyshev (nx % 4 == 0), one-node-per-thread CG (odd nx), one-node-per-thread Chebyshev
@pytest.mark.parametrize("solver,shape", [("cheb", (32, 24, 1)), ("cg", (31, 24, 1)), ("cheb", (15, 9, 4))])
def test_barrier_wait_runs_out_and_the_handle_recovers(solver, shape):
    wl = I.hh_sheet_32().with_mesh(*shape)
    s = P.Solver.from_workload(wl, solver=solver, cg_maxit=2000)
    m = O.Monodomain(wl)
    rng = np.random.default_rng(3)
    b = rng.normal(size=wl.n_nodes)
    g = 0.2
    want = m.solve_shifted(g, b, method=O.SOLVE_DCT)
    bd = torch.from_numpy(b).cuda()

    s.debug_barrier(0, 2000)                      # block 0 skips its first arrival; waits give up after 2 ms
    xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    with pytest.raises(P.EsdcError) as e:
        s.diffusion_solve(g, bd, xd)
    assert e.value.code == TIMEOUT
    assert time.perf_counter() - t0 < 0.5         # the 2 ms limit, not the 1 s default

    s.debug_barrier(-1)                           # normal waits again: the same handle solves correctly
    xd = torch.zeros(wl.n_nodes, dtype=torch.float64, device="cuda")
    assert s.diffusion_solve(g, bd, xd) >= 1
    assert rel(xd.cpu().numpy(), want) < 50 * (1 + 12 * g / wl.h**2) * 1e-14


def test_sweep_reports_timeout_then_steps_normally():
    wl = I.hh_sheet_32().with_mesh(16, 12, 1)
    M, K = wl.M, wl.K
    s = P.Solver.from_workload(wl, M_max=M, solver="cheb")
    y0 = I.random_state(wl, seed=9)

    def dev(y):
        t = s.new_state()
        t[:, :wl.n_nodes] = torch.from_numpy(np.ascontiguousarray(y))
        return t

    s.debug_barrier(0, 2000)
    yd = dev(y0)
    s.sweep(yd, 0.5, wl.dt, M, K)
    assert s.residual()[0] == TIMEOUT
    s.debug_barrier(-1)
    yd = dev(y0)
    s.sweep(yd, 0.5, wl.dt, M, K)
    assert s.residual()[0] == 0
    torch.cuda.synchronize()
    got = yd[:, :wl.n_nodes].cpu().numpy()
    want, _, _, _ = O.Monodomain(wl).step(y0, 0.5, wl.dt, M, K)
    assert rel(got[0], want[0]) < 1e-12
