"""Ragged batches (esdc_batch_*): every tissue of a batch against the FP64 oracle
run on that tissue alone, and bit-for-bit identity of the batched results with
the same tissues stepped one at a time, across launch shapes, with and without
the recorded CUDA graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
import paper_2405_19994_gb300 as P  # noqa: E402
from paper_2405_19994_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    P.lib()


def small_batch():
    """Seven ragged tissues: odd and even sides, a 1D strip, one single-tile tissue,
    and one spanning several tiles; stimulus patches at seeded positions."""
    wls = I.hh_batch(n=5, seed=11, side=(3, 41), sigma=(0.05, 0.3), patch=4)
    wls.append(I.hh_batch(n=1, seed=12, side=(37, 37))[0].with_mesh(37, 1, 1))      # 1D strip
    wls.append(I.hh_batch(n=1, seed=13, side=(48, 48))[0])                          # 2304 nodes, 5 tiles
    return wls


def run_batch(wls, steps, shape=None, graph=True, t0=0.0, solver="auto", persistent=None, want_iters=False,
              fuse_node1=True):
    b = P.Batch.from_workloads(wls, M_max=3, solver=solver, fuse_node1=fuse_node1)
    if shape:
        b.set_shape(*shape)
    if persistent:
        b.set_persistent(True, *persistent)
    b.set_graph(graph)
    y = b.new_state()
    b.init_state(y, -75.0)
    w0 = wls[0]
    t = t0
    for _ in range(steps):
        b.sweep(y, t, w0.dt, w0.M, w0.K)
        t += w0.dt
    rc, r, ym = b.residual()
    assert rc == 0, P.esdc.ERRORS.get(rc)
    torch.cuda.synchronize()
    out = [b.tissue(y, k).cpu().numpy().copy() for k in range(len(wls))]
    graph_used = (b.graph_active(), b.graph_error())
    iters = b.stats(wls[0].K, wls[0].M).copy() if want_iters else None
    b.close()
    if want_iters:
        return out, r, graph_used, iters
    return out, r, graph_used


@pytest.mark.parametrize("solver", ["auto", "cg"])
def test_batch_matches_oracle_per_tissue(solver):
    wls = small_batch()
    steps = 8
    got, res, _ = run_batch(wls, steps, solver=solver)
    for k, w in enumerate(wls):
        m = O.Monodomain(w)
        y = m.init_state()
        t = 0.0
        for _ in range(steps):
            y, st, _, _ = m.step(y, t, w.dt, w.M, w.K)
            t += w.dt
        err = np.abs(got[k][0] - y[0]).max() / np.abs(y[0]).max()
        assert err < 1e-12, (k, w.name, err)
        assert np.abs(got[k][1:] - y[1:]).max() < 1e-12, (k, w.name)


@pytest.mark.parametrize("persistent", [None, (512, 128)])
def test_batch_fused_node1_equals_separate_launches(persistent):
    # node 1 of each sweep inside the set-up / final-evaluation launch (or, in
    # the persistent step, phase) against its own: the same bits
    wls = small_batch()
    a, ra, _, ia = run_batch(wls, 5, persistent=persistent, want_iters=True)
    b, rb, _, ib = run_batch(wls, 5, persistent=persistent, want_iters=True, fuse_node1=False)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(ia, ib)


@pytest.mark.parametrize("solver", ["auto", "cg"])
def test_batch_bitwise_equals_one_at_a_time(solver):
    wls = small_batch()
    steps = 6
    batched, _, _ = run_batch(wls, steps, solver=solver)
    for k, w in enumerate(wls):
        alone, _, _ = run_batch([w], steps, solver=solver)
        assert np.array_equal(batched[k], alone[0]), (k, w.name)


def test_batch_chebyshev_degenerate_tissues():
    """A single node (the operator is the identity: an interval of no width), a
    four-node strip and a thin slab in one batch, each against the oracle."""
    base = I.hh_batch(n=1, seed=21, side=(12, 12))[0]
    wls = [base.with_mesh(1, 1, 1), base.with_mesh(4, 1, 1), base.with_mesh(9, 5, 2), base]
    steps = 6
    got, _, _ = run_batch(wls, steps)
    for k, w in enumerate(wls):
        m = O.Monodomain(w)
        y = m.init_state()
        t = 0.0
        for _ in range(steps):
            y, _, _, _ = m.step(y, t, w.dt, w.M, w.K)
            t += w.dt
        assert np.abs(got[k] - y).max() < 1e-12 * max(1.0, np.abs(y).max()), (k, w.nx, w.ny, w.nz)


@pytest.mark.parametrize("shape", [(1, 512, 1), (2, 256, 2), (4, 256, 1)])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_results_independent_of_launch_shape_and_graph(shape, graph):
    wls = small_batch()
    ref, _, _ = run_batch(wls, 4)
    got, _, used = run_batch(wls, 4, shape=shape, graph=graph)
    for k in range(len(wls)):
        assert np.array_equal(ref[k], got[k]), (shape, graph, k)
    if not graph:
        assert not used[0]
    else:
        assert used[0], "the step was not recorded in a CUDA graph: " + used[1]


# ---------------------------------------------------------------- one persistent launch per step

@pytest.mark.parametrize("threads,tile,graph", [(512, 32, True), (512, 128, False), (256, 512, True),
                                                (512, 2048, True), (256, 64, False)])
def test_persistent_step_bitwise_equals_launch_sequence(threads, tile, graph):
    """The whole step in one cooperative kernel (set-up, node phases, the
    Chebyshev solves of all tissues, residual) against the launch sequence:
    identical bit for bit, solve iteration counts included, whatever the block
    size, node tile or graph."""
    wls = small_batch()
    ref, rr, _, it_ref = run_batch(wls, 5, want_iters=True)
    got, rg, used, it = run_batch(wls, 5, graph=graph, persistent=(threads, tile), want_iters=True)
    for k in range(len(wls)):
        assert np.array_equal(ref[k], got[k]), (threads, tile, graph, k)
    assert np.array_equal(rr, rg)
    assert np.array_equal(it_ref, it)
    assert used[0] == graph, used[1]


def test_persistent_qpar_and_tau_bitwise_equal_launch_sequence():
    """Q^par (set-up from the iterate) and the FAS sweep with tau run through the
    persistent kernel exactly as through the launch sequence."""
    P_, iters = 4, 3
    w, m, y0, t0 = qpar_setup(P_)
    outs = []
    for persist in (False, True):
        b = P.Batch.from_workloads([w] * P_, M_max=w.M)
        if persist:
            b.set_persistent(True, 512, 128)
        yin, yout = b.new_state(), b.new_state()
        b.tissue(yin, 0).copy_(torch.from_numpy(y0))
        b.qpar(yin, yout, t0, w.dt, w.M, iters)
        assert b.residual()[0] == 0
        outs.append(yout.clone())
        b.close()
    assert torch.equal(outs[0], outs[1])


def test_persistent_rejected_with_cg():
    b = P.Batch.from_workloads(small_batch()[:2], M_max=3, solver="cg")
    with pytest.raises(P.EsdcError) as e:
        b.set_persistent(True)
    assert e.value.code == -6
    b.close()


def test_batch_matches_single_tissue_solver():
    """Against esdc_sweep on each tissue (a different CG reduction order, so the
    agreement is to the CG tolerance rather than bitwise)."""
    wls = small_batch()
    steps = 5
    got, _, _ = run_batch(wls, steps)
    for k, w in enumerate(wls):
        s = P.Solver.from_workload(w, M_max=3)
        y = s.new_state()
        s.init_state(y, w.V0)
        t = 0.0
        for _ in range(steps):
            s.sweep(y, t, w.dt, w.M, w.K)
            t += w.dt
        assert s.residual()[0] == 0
        torch.cuda.synchronize()
        ys = y[:, :w.n_nodes].cpu().numpy()
        assert np.abs(got[k] - ys).max() < 1e-11 * max(1.0, np.abs(ys).max()), k
        s.close()


def test_batch_per_tissue_start_times_and_stimulus_windows():
    """Tissues at different t_n: a tissue whose window has passed is not stimulated."""
    wls = small_batch()[:3]
    b = P.Batch.from_workloads(wls, M_max=3)
    y = b.new_state()
    b.init_state(y, -75.0)
    w0 = wls[0]
    tv = np.array([0.0, 5.0, 0.5])
    for _ in range(4):
        b.sweep(y, tv, w0.dt, w0.M, w0.K)
        tv = tv + w0.dt
    assert b.residual()[0] == 0
    torch.cuda.synchronize()
    for k, w in enumerate(wls):
        m = O.Monodomain(w)
        yo = m.init_state()
        t = [0.0, 5.0, 0.5][k]
        for _ in range(4):
            yo, _, _, _ = m.step(yo, t, w.dt, w.M, w.K)
            t += w.dt
        got = b.tissue(y, k).cpu().numpy()
        assert np.abs(got[0] - yo[0]).max() < 1e-12 * np.abs(yo[0]).max(), k
    b.close()


def test_batch_tuner_keeps_results():
    wls = small_batch()
    ref, _, _ = run_batch(wls, 3)
    b = P.Batch.from_workloads(wls, M_max=3)
    scratch = b.new_state()
    w0 = wls[0]
    b.tune(scratch, -75.0, 0.0, w0.dt, w0.M, w0.K, reps=1)
    waves, threads, blocks = b.shape()
    assert waves in (1, 2, 4) and threads in (256, 512) and blocks >= 1
    y = b.new_state()
    b.init_state(y, -75.0)
    t = 0.0
    for _ in range(3):
        b.sweep(y, t, w0.dt, w0.M, w0.K)
        t += w0.dt
    assert b.residual()[0] == 0
    torch.cuda.synchronize()
    for k in range(len(wls)):
        assert np.array_equal(b.tissue(y, k).cpu().numpy(), ref[k]), k
    b.close()


@pytest.mark.parametrize("solver", ["auto", "cg"])
def test_batch_cg_maxit_reported_per_batch(solver):
    wls = small_batch()[:2]
    b = P.Batch.from_workloads(wls, M_max=3, cg_maxit=1, solver=solver)
    y = b.new_state()
    b.init_state(y, -75.0)
    w0 = wls[0]
    b.sweep(y, 0.0, w0.dt, w0.M, w0.K)
    rc, _, _ = b.residual()
    assert rc == -3
    it = b.stats(w0.K, w0.M)
    assert it.max() <= 1
    b.close()


# ---------------------------------------------------------------- Q^par: time slices as the batch

def qpar_setup(P=4, nx=10, ny=8):
    w = I.hh_sheet_32().with_mesh(nx, ny, 1)
    m = O.Monodomain(w)
    y0, t0 = m.init_state(), 0.0
    for _ in range(16):                               # a state inside the stimulus window, mid-upstroke
        y0, _, _, _ = m.step(y0, t0, w.dt, w.M, w.K)
        t0 += w.dt
    return w, m, y0, t0


def test_qpar_matches_oracle():
    P_, iters = 4, 3
    w, m, y0, t0 = qpar_setup(P_)
    b = P.Batch.from_workloads([w] * P_, M_max=w.M)
    yin, yout = b.new_state(), b.new_state()
    b.tissue(yin, 0).copy_(torch.from_numpy(y0))
    b.qpar(yin, yout, t0, w.dt, w.M, iters)
    assert b.residual()[0] == 0
    Z = m.qpar(y0, t0, w.dt, P_, w.M, iters)
    torch.cuda.synchronize()
    for p in range(P_):
        got = b.tissue(yout, p).cpu().numpy()
        want = Z[p, w.M - 1]
        assert np.abs(got[0] - want[0]).max() < 1e-12 * np.abs(want[0]).max(), p
        assert np.abs(got[1:] - want[1:]).max() < 1e-12, p
    b.close()


def test_qpar_bitwise_equals_looped_slices():
    P_, iters = 4, 3
    w, m, y0, t0 = qpar_setup(P_)
    b = P.Batch.from_workloads([w] * P_, M_max=w.M)
    yin, yout = b.new_state(), b.new_state()
    b.tissue(yin, 0).copy_(torch.from_numpy(y0))
    b.qpar(yin, yout, t0, w.dt, w.M, iters)
    assert b.residual()[0] == 0
    torch.cuda.synchronize()
    singles = [P.Batch.from_workloads([w], M_max=w.M) for _ in range(P_)]
    yi = [s.new_state() for s in singles]
    yo = [s.new_state() for s in singles]
    y0d = torch.from_numpy(y0).cuda()
    ends = None
    for k in range(iters):
        for p, s in enumerate(singles):
            src = y0d if (p == 0 or ends is None) else ends[p - 1]
            s.tissue(yi[p], 0).copy_(src)
            s.sweep_from(yi[p], yo[p], t0 + p * w.dt, w.dt, w.M, 1, from_iterate=k > 0)
        ends = [s.tissue(yo[p], 0).clone() for p, s in enumerate(singles)]
    for p, s in enumerate(singles):
        assert s.residual()[0] == 0
        assert torch.equal(b.tissue(yout, p), s.tissue(yo[p], 0)), p
        s.close()
    b.close()


def test_qpar_one_slice_is_k_sweeps_of_the_step():
    w, m, y0, t0 = qpar_setup(1)
    b = P.Batch.from_workloads([w], M_max=w.M)
    yin, yout = b.new_state(), b.new_state()
    b.tissue(yin, 0).copy_(torch.from_numpy(y0))
    b.qpar(yin, yout, t0, w.dt, w.M, w.K)
    want, _, _, _ = m.step(y0, t0, w.dt, w.M, w.K)
    assert b.residual()[0] == 0
    got = b.tissue(yout, 0).cpu().numpy()
    assert np.abs(got[0] - want[0]).max() < 1e-12 * np.abs(want[0]).max()
    b.close()


# ---------------------------------------------------------------- FAS: tau-corrected sweeps, two-level Algorithm HSDC

def test_sweep_with_tau_matches_oracle():
    w, m, y0, t0 = qpar_setup(1)
    M = w.M
    rng = np.random.default_rng(17)
    _, _, col, _ = m.step(y0, t0, w.dt, M, 2, want_colloc=True)
    tau = 1e-3 * rng.normal(size=col.shape) * np.abs(col).max(axis=(0, 2), keepdims=True)
    b = P.Batch.from_workloads([w], M_max=M)
    yin, yout = b.new_state(), b.new_state()
    b.tissue(yin, 0).copy_(torch.from_numpy(y0))
    Y = b.iterate(M)
    for j in range(M):
        Y[j, :, :w.n_nodes] = torch.from_numpy(col[j])
    td = torch.zeros((M, b.n_state, b.ld), dtype=torch.float64, device="cuda")
    td[:, :, :w.n_nodes] = torch.from_numpy(tau)
    tv = np.array([t0])
    P.lib().esdc_batch_sweep_ex(b._b, yin.data_ptr(), yout.data_ptr(), td.data_ptr(),
                                tv.ctypes.data_as(E_D()), w.dt, M, 2, 1, 0, torch.cuda.current_stream().cuda_stream)
    assert b.residual()[0] == 0
    want, _, wcol, _ = m.step(y0, t0, w.dt, M, 2, want_colloc=True, colloc_in=col, tau=tau)
    got = b.iterate(M)[:, :, :w.n_nodes].cpu().numpy()
    assert np.abs(got - wcol).max() < 1e-12 * np.abs(wcol).max()
    b.close()


def E_D():
    import ctypes
    return ctypes.POINTER(ctypes.c_double)


@pytest.mark.parametrize("iters", [1, 3])
def test_hsdc2_matches_oracle(iters):
    P_, M1, M2 = 4, 3, 2
    w, m, y0, t0 = qpar_setup(P_)
    fine = P.Batch.from_workloads([w] * P_, M_max=M1)
    coarse = [P.Batch.from_workloads([w], M_max=M2) for _ in range(P_)]
    yin, yout = fine.new_state(), fine.new_state()
    fine.tissue(yin, 0).copy_(torch.from_numpy(y0))
    P.esdc.hsdc2(fine, coarse, yin, yout, t0, w.dt, M1, M2, iters)
    assert fine.residual()[0] == 0
    Z = m.hsdc2(y0, t0, w.dt, P_, M1, M2, iters)
    Y = fine.iterate(M1)
    for p in range(P_):
        o = int(fine.offsets[p])
        got = Y[:, :, o:o + w.n_nodes].cpu().numpy()
        assert np.abs(got - Z[p]).max() < 1e-12 * np.abs(Z[p]).max(), p
        assert np.array_equal(fine.tissue(yout, p).cpu().numpy(), got[M1 - 1]), p
    for c in coarse:
        c.close()
    fine.close()


def test_hsdc2_converges_to_sequential_collocation():
    P_, M1, M2 = 4, 3, 2
    w, m, y0, t0 = qpar_setup(P_)
    fine = P.Batch.from_workloads([w] * P_, M_max=M1)
    coarse = [P.Batch.from_workloads([w], M_max=M2) for _ in range(P_)]
    yin, yout = fine.new_state(), fine.new_state()
    fine.tissue(yin, 0).copy_(torch.from_numpy(y0))
    P.esdc.hsdc2(fine, coarse, yin, yout, t0, w.dt, M1, M2, 14)
    y, t = y0, t0
    for p in range(P_):
        yn, _, col, _ = m.step(y, t, w.dt, M1, 60, want_colloc=True)
        got = fine.tissue(yout, p).cpu().numpy()
        assert np.abs(got - yn).max() < 1e-11 * np.abs(yn).max(), p
        y, t = yn, t + w.dt
    for c in coarse:
        c.close()
    fine.close()


@pytest.mark.parametrize("iters", [1, 3])
def test_hsdc_three_levels_matches_oracle(iters):
    P_, Ms = 4, (3, 2, 1)
    w, m, y0, t0 = qpar_setup(P_)
    levels = [P.Batch.from_workloads([w] * P_, M_max=Ms[0]), P.Batch.from_workloads([w] * P_, M_max=Ms[1])]
    coarse = [P.Batch.from_workloads([w], M_max=Ms[2]) for _ in range(P_)]
    fine = levels[0]
    yin, yout = fine.new_state(), fine.new_state()
    fine.tissue(yin, 0).copy_(torch.from_numpy(y0))
    P.esdc.hsdc(levels, coarse, yin, yout, t0, w.dt, Ms, iters)
    assert fine.residual()[0] == 0
    Z = m.hsdc(y0, t0, w.dt, P_, Ms, iters)
    Y = fine.iterate(Ms[0])
    for p in range(P_):
        o = int(fine.offsets[p])
        got = Y[:, :, o:o + w.n_nodes].cpu().numpy()
        assert np.abs(got - Z[p]).max() < 1e-12 * np.abs(Z[p]).max(), p
        assert np.array_equal(fine.tissue(yout, p).cpu().numpy(), got[Ms[0] - 1]), p
    for b in coarse + levels:
        b.close()


def test_hsdc_three_levels_converges_to_sequential_collocation():
    P_, Ms = 4, (3, 2, 1)
    w, m, y0, t0 = qpar_setup(P_)
    levels = [P.Batch.from_workloads([w] * P_, M_max=Ms[0]), P.Batch.from_workloads([w] * P_, M_max=Ms[1])]
    coarse = [P.Batch.from_workloads([w], M_max=Ms[2]) for _ in range(P_)]
    fine = levels[0]
    yin, yout = fine.new_state(), fine.new_state()
    fine.tissue(yin, 0).copy_(torch.from_numpy(y0))
    P.esdc.hsdc(levels, coarse, yin, yout, t0, w.dt, Ms, 16)
    y, t = y0, t0
    for p in range(P_):
        yn, _, _, _ = m.step(y, t, w.dt, Ms[0], 60)
        got = fine.tissue(yout, p).cpu().numpy()
        assert np.abs(got - yn).max() < 1e-11 * np.abs(yn).max(), p
        y, t = yn, t + w.dt
    for b in coarse + levels:
        b.close()


def test_hsdc_rejects_bad_levels():
    P_ = 2
    w, m, y0, t0 = qpar_setup(P_)
    fine = P.Batch.from_workloads([w] * P_, M_max=3)
    mid = P.Batch.from_workloads([w] * P_, M_max=1)                 # M_max below its level's M
    coarse = [P.Batch.from_workloads([w], M_max=1) for _ in range(P_)]
    yin, yout = fine.new_state(), fine.new_state()
    for Ms, levels in (((3, 3, 1), [fine, mid]), ((3, 2, 1), [fine, mid]), ((3,), [fine])):
        with pytest.raises(P.EsdcError) as e:
            P.esdc.hsdc(levels, coarse, yin, yout, t0, w.dt, Ms, 1)
        assert e.value.code == -1
    for b in coarse + [fine, mid]:
        b.close()


@pytest.mark.slow
@pytest.mark.slow
def test_full_batch_persistent_matches_oracle():
    """The full 64-tissue batch (5.1M nodes) with one persistent launch per step
    (recorded graph): after 3 steps from rest, the three smallest tissues
    against the oracle, element by element."""
    wls = I.hh_batch()
    w0 = wls[0]
    b = P.Batch.from_workloads(wls, M_max=w0.M)
    b.set_persistent(True, 512, 128)
    y = b.new_state()
    b.init_state(y, w0.V0)
    t = 0.0
    for _ in range(3):
        b.sweep(y, t, w0.dt, w0.M, w0.K)
        t += w0.dt
    assert b.residual()[0] == 0
    assert b.graph_active()
    torch.cuda.synchronize()
    for k in sorted(range(len(wls)), key=lambda j: wls[j].n_nodes)[:3]:
        w = wls[k]
        m = O.Monodomain(w)
        yo = m.init_state()
        to = 0.0
        for _ in range(3):
            yo, _, _, _ = m.step(yo, to, w.dt, w.M, w.K)
            to += w.dt
        got = b.tissue(y, k).cpu().numpy()
        assert np.abs(got - yo).max() < 1e-12 * max(1.0, np.abs(yo).max()), (k, w.name)
    b.close()


def test_full_batch_in_bench_configuration_matches_oracle():
    """The 64-tissue batch of the batching form at full size (5.1M nodes), in the
    launch configuration the bench ends up with (recorded graph, 4 node waves,
    256-thread solve blocks, 2 per SM): after 3 steps from rest, the three
    smallest tissues against the oracle run on each alone, element by element."""
    wls = I.hh_batch()
    w0 = wls[0]
    b = P.Batch.from_workloads(wls, M_max=w0.M)
    b.set_shape(4, 256, 2)
    b.set_graph(True)
    y = b.new_state()
    b.init_state(y, w0.V0)
    t = 0.0
    for _ in range(3):
        b.sweep(y, t, w0.dt, w0.M, w0.K)
        t += w0.dt
    assert b.residual()[0] == 0
    assert b.graph_active()
    torch.cuda.synchronize()
    for k in sorted(range(len(wls)), key=lambda j: wls[j].n_nodes)[:3]:
        w = wls[k]
        m = O.Monodomain(w)
        yo = m.init_state()
        to = 0.0
        for _ in range(3):
            yo, _, _, _ = m.step(yo, to, w.dt, w.M, w.K)
            to += w.dt
        got = b.tissue(y, k).cpu().numpy()
        assert np.abs(got - yo).max() < 1e-12 * max(1.0, np.abs(yo).max()), (k, w.name)
    b.close()


def test_batch_graph_rerecorded_after_setup_table_refill():
    # A recorded step points at the set-up coefficient table of its (M, dt).
    # Record a step from the stored iterate at dt0 (the batch's second graph),
    # then let plain steps at five
    # other step sizes refill all four table slots, then repeat the first call
    # unchanged: its graph must be recorded again against the rebuilt table.
    # The same sequence without graphs gives the reference bits.
    wls = small_batch()
    dt0 = wls[0].dt
    others = [0.011, 0.013, 0.017, 0.019, 0.023]

    def run(graph):
        b = P.Batch.from_workloads(wls, M_max=3)
        b.set_graph(graph)
        y = b.new_state()
        y2 = b.new_state()
        b.init_state(y, -75.0)
        b.sweep(y, 0.0, dt0, 3, 2)
        b.sweep_from(y, y2, 0.0, dt0, 3, 1, True)
        for dt in others:
            b.sweep(y, 0.0, dt, 3, 1)
            b.sweep(y, 0.0, dt, 3, 1)
        b.sweep_from(y, y2, 0.0, dt0, 3, 1, True)
        assert b.residual()[0] == 0
        used = b.graph_active()
        torch.cuda.synchronize()
        out = [b.tissue(y2, k).cpu().numpy().copy() for k in range(len(wls))]
        b.close()
        return out, used

    got, used = run(True)
    want, _ = run(False)
    assert used
    for x, w in zip(got, want):
        np.testing.assert_array_equal(x, w)
