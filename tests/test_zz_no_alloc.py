"""The allocation-free diffusion solve (esdc_diffusion_solve_static) against the
handle-based one (esdc_diffusion_solve), through the C ABI.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes alone in a fresh
process and after the other tests (the shared scratch array is cleared by each
call where it must start at zero)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(48, 40, 9), (47, 40, 9)])
def test_static_scratch_solve_matches_handle_solve(shape):
    """48 x 40 x 9 takes the quad CG (nx a multiple of 4); 47 x 40 x 9 the
    one-node-per-thread CG, which odd, unaligned and fourth-order callers reach.
    Both against the handle's solve run the same way and against the oracle's
    exact DCT-II solve, on two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import paper_2405_19994_gb300 as P
    from oracle import oracle as O
    from paper_2405_19994_gb300 import esdc as E
    from paper_2405_19994_gb300 import inputs as I

    L = P.lib()
    wl = I.hh_sheet_32().with_mesh(*shape)
    tol, maxit = 1e-14, 500
    # the static solve runs the Jacobi-PCG: compare with the handle's solve run the same way
    s = P.Solver.from_workload(wl, tol_cg=tol, cg_maxit=maxit, solver="cg")
    m = O.Monodomain(wl)
    mesh = E.esdc_mesh(wl.dim, wl.nx, wl.ny, wl.nz, wl.h)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(12)
    for call, g in enumerate((0.031, 0.2)):             # two calls in a row
        bh = rng.normal(size=wl.n_nodes)
        b = torch.from_numpy(bh).cuda()
        x0 = torch.from_numpy(rng.normal(size=wl.n_nodes)).cuda()
        x_ref = x0.clone()
        it_ref = s.diffusion_solve(g, b, x_ref)
        x = x0.clone()
        it = C.c_int(-1)
        rc = L.esdc_diffusion_solve_static(C.byref(mesh), g, b.data_ptr(), x.data_ptr(), tol, maxit, 1,
                                           C.byref(it), stream)
        assert rc == 0, (call, rc)
        # both are the same CG to ||r|| <= 1e-14 ||b||: the solutions agree to
        # kappa * tol with kappa = 1 + 12 g / h^2, and so does each with the exact solve
        bound = 50 * (1 + 12 * g / wl.h**2) * tol
        err = (x - x_ref).abs().max().item() / x_ref.abs().max().item()
        assert err <= bound, (call, err)
        assert it.value == it_ref, (call, it.value, it_ref)
        want = m.solve_shifted(g, bh, method=O.SOLVE_DCT)
        got = x.cpu().numpy()
        assert np.abs(got - want).max() / np.abs(want).max() <= bound, call

    # a mesh beyond the fixed scratch is refused before any GPU work
    big = E.esdc_mesh(3, 128, 128, 17, 0.2)
    rc = L.esdc_diffusion_solve_static(C.byref(big), 0.1, b.data_ptr(), x.data_ptr(), tol, maxit, 1, None, stream)
    assert rc == -8
