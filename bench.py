#!/usr/bin/env python3
"""ES-SDC (HSDC) benchmark on one GB300.

Workload (the headline configuration): 128x128x32 slab (524,288 nodes),
h = 0.2 mm, seeded 19-state synthetic stiff ionic model, planar stimulus at
x = 0 for t < 1 ms, M = 4 Radau IIA nodes, K = 6 sweeps, dt = 0.05 ms, FP64.
A bench "step" is one HSDC time step: set-up, K sweeps over the M nodes (fused
ionic/quadrature kernel + CG diffusion solve each) and the collocation residual.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is node-updates/s (one mesh node advanced by
one dt), device-timed with CUDA events over K steps.  Before them the run goes,
untimed, from rest through the stimulus (t < 1 ms) and --pre-steps (100) steps
after it, then W warm-up steps, so the timed window sees a propagating wave
(config.window_ms).  ``--impl reference`` times the FP64 CPU oracle on this
host instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ES-SDC node-updates/s and s per simulated ms at stated V-error; % roofline"
UNIT = "node-updates/s"

# Work per unit, used for the roofline of the dominant kernel.
#  node kernel (SYN19, M = 4), per mesh node and sweep: the M + 1 launches of a
#  sweep are node 1 (quadrature only), nodes 2..M (ionic evaluation + quadrature)
#  and the final evaluation at node M.  FP64 flops (FMA = 2) counted by ncu
#  (thread-level DFMA/DADD/DMUL) over the 5 launches of one sweep, with the gate
#  functions evaluated from their V table (degree 3 on 1/128 mV intervals, the
#  pairs (Lambda, -Lambda w_inf)):
#  191.0 + 3 x 483.7 + 271.7 = 1913.8 flops per node per sweep
#  (profiles/classes_syn19_slab_128x128x16.md).
#  Algorithmic bytes per node: node 1 reads 158 / writes 20 doubles, nodes 2..M
#  204 / 20, the final evaluation 63 / 20 -> 7464 B per sweep.  DRAM traffic
#  per node and launch measured by ncu, keyed by (M, node 1 fused), in
#  NODE_DRAM_BYTES_PER_LAUNCH_MEASURED (profiles/classes_syn19_slab_128x128x16.md).
#  cg (per mesh node and iteration): [A] z (stencil), p, q -> p, q;
#  [B] q, r, x, p -> x, r, z: 12 doubles = 96 B, plus 8 doubles per solve.
#  Node 1 of each sweep (quadrature only: 96.0 FP64 instructions, 191.0 flops,
#  158 + 20 doubles) runs inside the launch before it (the set-up, or the
#  previous sweep's final evaluation): a step has K M node launches, and the
#  set-up class carries the first sweep's node 1.
NODE_FLOPS_PER_SWEEP = {4: 1913.8}
NODE_BYTES_PER_SWEEP = {4: 7464}
NODE1 = {"fp64_ops": 96.0, "flops": 191.0, "bytes": 1424}
#  ncu, 262,144 nodes, node 1 fused, 6 blocks per SM: 18 x 1825.1 + 5 x 1748.0 +
#  431.3 B per step over 24 launches.
NODE_DRAM_BYTES_PER_LAUNCH_MEASURED = {(4, True): 1751.0}
CG_BYTES_PER_NODE_ITER = 96
CG_BYTES_PER_NODE_SETUP = 64
# FP64 peak: 152 SMs x 2 FP64 FMA per clock per SM x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64 issue peak: 152 SMs x 2 FP64 instructions (thread level) per clock x 2.07 GHz.
FP64_ISSUE_PEAK = 152 * 2 * 2.07e9

# Work per mesh node of each kernel class of one step (M = 4, SYN19): FP64
# instructions (thread-level DFMA + DADD + DMUL, counted by ncu on the
# 128x128x16 slab, profiles/classes_syn19_slab_128x128x16.md) and the bytes the
# method streams.  Set-up: the coefficient tables (from their table in z) and
# one ionic evaluation per step; node: per sweep (M + 1 launches); DCT solve: four transform passes
# and the tridiagonal z solve; Chebyshev and CG: per iteration; residual: per
# step.
CLASS_FP64_OPS = {"setup": 903.1, "node_sweep": 1114.8, "dct_solve": 54.3, "cheb_iter": 12.2, "cg_iter": 15.0,
                  "residual": 551.0}
CLASS_BYTES = {"setup": 3256.0, "node_sweep": 7464.0, "dct_solve": 120.0, "cheb_iter": 48.0, "cg_iter": 96.0,
               "residual": 2904.0}


def class_work(solver_kind: str, K: int, it_mean: float, M: int = 4, fused: bool = True) -> dict:
    """(FP64 instructions, bytes) per node and step of each kernel class; with
    `fused`, the first sweep's node 1 belongs to the set-up launch."""
    solves = M * K
    if solver_kind == "dct":
        sv = (CLASS_FP64_OPS["dct_solve"] * solves, CLASS_BYTES["dct_solve"] * solves)
    else:
        sv = (CLASS_FP64_OPS["cheb_iter"] * it_mean * solves, CLASS_BYTES["cheb_iter"] * it_mean * solves)
    n1 = (NODE1["fp64_ops"], NODE1["bytes"]) if fused else (0.0, 0.0)
    return {"setup": (CLASS_FP64_OPS["setup"] + n1[0], CLASS_BYTES["setup"] + n1[1]),
            "node": (CLASS_FP64_OPS["node_sweep"] * K - n1[0], CLASS_BYTES["node_sweep"] * K - n1[1]),
            "cg": sv,
            "residual": (CLASS_FP64_OPS["residual"], CLASS_BYTES["residual"])}


def DCT_KERNELS_PER_SOLVE(wl) -> int:
    """Kernel launches of one DCT-II solve of the second-order stencil: the
    forward and inverse x transforms (nx > 1), then either the fused y-z kernel
    (the library's rule: ny a power of two >= 16, nz >= 2, and the y-z slab,
    its z factors and the twiddles within one block's 200 KB of shared memory
    and 1024 threads) or the y transforms (ny > 1) and the z solve."""
    ny, nz = wl.ny, wl.nz
    pairs, g = (nz + 1) // 2, min(ny // 4, 256)
    fused = (ny >= 16 and ny & (ny - 1) == 0 and nz >= 2 and (pairs * g + 31) // 32 * 32 <= 1024
             and (ny + 2 * pairs * (ny + 1)) * 16 + 2 * nz * ny * 8 <= 200 * 1024)
    return 2 * (wl.nx > 1) + (1 if fused else 2 * (ny > 1) + 1)


def _peaks():
    p = {"hbm_gbs": None, "source": None}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        p["hbm_gbs"] = d.get("hbm_gbs")
        p["source"] = "measured"
    if not p["hbm_gbs"]:
        p["hbm_gbs"], p["source"] = 6800.0, "fallback"
    return p


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region (200 ms period)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, pg=None) -> float:
    """The slowest rank's time: every rank passes its own, all get the maximum."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(units_per_rank: float, world_size: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world_size / (ms * 1e-3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on this host's cores.  Each step is a
    bounded sample of the workload: one HSDC step of the 128x128x2 sub-slab
    (32,768 nodes, the same per-node work)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2405_19994_gb300 import inputs as I
    wl = I.syn19_slab()
    sub = wl.with_mesh(wl.nx, wl.ny, 2)
    m = oracle.Monodomain(sub)
    y = m.init_state()
    t = 0.0
    for n in range(args.warmup):
        y, _, _, _ = m.step(y, t, wl.dt, wl.M, wl.K)
        t += wl.dt
    t0 = time.perf_counter()
    for n in range(args.steps):
        y, _, _, _ = m.step(y, t, wl.dt, wl.M, wl.K)
        t += wl.dt
    el = time.perf_counter() - t0
    value = sub.n_nodes * args.steps / el
    cores = oracle.oracle.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "sample": "128x128x2 sub-slab (32768 nodes)", "M": wl.M,
                   "K": wl.K, "dt_ms": wl.dt, "model": "syn19 (seed 20240530)"},
        "s_per_sim_ms": (el / args.steps) / wl.dt * (wl.n_nodes / sub.n_nodes),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "HSDC steps of the 128x128x2 sub-slab of the workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _strip_dt8_error(wl, t_w, n_window, dt):
    """Time-discretisation error of the window [t_w, t_w + n_window dt] from the
    oracle on the 128x1x1 strip: the headline slab's planar wave (stimulus on
    the whole x = 0 face, uniform initial state, zero-flux faces) does not vary
    in y or z, so the strip carries the slab's solution.  The strip runs at dt
    from rest to t_w, then over the window once at dt and once at dt/8 from that
    state.  Returns (V(dt), V(dt/8)) at the window end and the oracle seconds."""
    import oracle
    strip = wl.with_mesh(wl.nx, 1, 1)
    m = oracle.Monodomain(strip)
    y = m.init_state()
    c0 = time.perf_counter()
    n_pre = int(round(t_w / dt))
    t = 0.0
    for _ in range(n_pre):
        y, _, _, _ = m.step(y, t, dt, wl.M, wl.K)
        t += dt
    ya, yb = y.copy(), y.copy()
    ta = tb = t
    for _ in range(n_window):
        ya, _, _, _ = m.step(ya, ta, dt, wl.M, wl.K)
        ta += dt
    for _ in range(8 * n_window):
        yb, _, _, _ = m.step(yb, tb, dt / 8, wl.M, wl.K)
        tb += dt / 8
    return ya[0], yb[0], time.perf_counter() - c0


def _rel(a, b):
    import numpy as np
    return float(np.abs(a - b).max() / np.abs(b).max())


def _rel2(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_ours(args):
    import numpy as np
    import torch
    import paper_2405_19994_gb300 as P
    from paper_2405_19994_gb300 import inputs as I

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    wl = I.syn19_slab()
    if args.nz and args.nz != wl.nz:         # smaller slab for profiler captures
        wl = wl.with_mesh(wl.nx, wl.ny, args.nz)
    M, K, dt = wl.M, wl.K, wl.dt
    N = wl.n_nodes
    solver = P.Solver.from_workload(wl, M_max=M, precision=args.precision, solver=args.solver)
    y = solver.new_state()
    solver.init_state(y, wl.V0)
    stream = torch.cuda.current_stream()
    # untimed: through the stimulus and args.pre_steps steps after it, so that
    # the timed window sees a propagating wave; then the warm-up steps
    n_stim = int(np.ceil(float(np.max(wl.t_off)) / dt - 1e-9))
    n_pre = n_stim + args.pre_steps
    t = 0.0
    for _ in range(n_pre + args.warmup):
        solver.sweep(y, t, dt, M, K)
        t += dt
    rc = solver.residual()[0]
    if rc != 0:
        raise RuntimeError(f"warm-up step failed with code {rc}")
    t_w = t
    y_w = y.clone()                           # state at the window start

    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    solver.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        solver.sweep(y, t, dt, M, K)
        t += dt
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    prof = solver.profile_read()
    solver.profile(False)
    clk = clocks.stop()
    rc, res_inf, y_inf, _ = solver.residual()
    cg_iters = solver.stats(K * M).tolist()
    if rc != 0:
        raise RuntimeError(f"timed step failed with code {rc}")
    ms = max_over_ranks(ms, pg)
    value = aggregate_value(N * args.steps, ws, ms)
    ms_step = ms / args.steps
    t_end = t
    V_end = y[0, :N].cpu().numpy().copy()     # V at the window end

    # ---- end to end: the same steps through the host-buffer entry point (H2D + step + D2H)
    ns, ld = solver.n_state, solver.ld
    y_host = torch.empty((ns, ld), dtype=torch.float64, pin_memory=True)
    y_host.copy_(y)
    torch.cuda.synchronize()
    n_e2e = max(1, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        solver.sweep_host(y_host, t, dt, M, K)
        t += dt
    e2e_s = time.perf_counter() - t0
    e2e_value = N * n_e2e * ws / e2e_s
    y.copy_(y_host.cuda())

    # ---- roofline of the dominant kernel class, and the FP64-issue fraction of every class
    peaks = _peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    per_launch_ms = {k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()}
    it_mean = sum(cg_iters) / max(len(cg_iters), 1)
    solver_kind = "dct" if solver.solver_in_use() == "dct" else "iter"
    roof = {"kernel": dom}
    node_launches_step = prof["node"][1] / args.steps if prof["node"][1] else 0
    fused = abs(node_launches_step - K * M) < 0.5                # node 1 inside the launch before it
    if dom == "node" and M in NODE_FLOPS_PER_SWEEP and args.precision == "fp64":
        # per launch: the node class's work per step over its launches per step
        flops = (NODE_FLOPS_PER_SWEEP[M] * K - (NODE1["flops"] if fused else 0.0)) * N / node_launches_step
        byts = (NODE_BYTES_PER_SWEEP[M] * K - (NODE1["bytes"] if fused else 0)) * N / node_launches_step
        ach = flops / (per_launch_ms["node"] * 1e-3) / 1e12
        # FP64 instructions (DFMA, DADD, DMUL alike) per launch over the issue peak:
        # the pipe's use whatever the instruction mix (flops count an FMA as 2)
        instr = (CLASS_FP64_OPS["node_sweep"] * K - (NODE1["fp64_ops"] if fused else 0.0)) * N / node_launches_step
        issue = instr / (per_launch_ms["node"] * 1e-3) / FP64_ISSUE_PEAK
        dram = NODE_DRAM_BYTES_PER_LAUNCH_MEASURED.get((M, fused))
        roof.update({"bound": "alu", "unit": "TFLOP/s", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                     "frac": ach / FP64_PEAK_TFLOPS,
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz; the "
                                    "library's FMA probe (bench.py --form peaks) measures 1.256 TFLOP/s",
                     "fp64_issue_frac": issue,
                     "launches_per_step": node_launches_step, "node1_fused": fused,
                     "traffic": dram * N if dram else None,
                     "algorithmic_bytes": byts,
                     "hbm_gbs": byts / (per_launch_ms["node"] * 1e-3) / 1e9,
                     "hbm_peak_gbs": peaks["hbm_gbs"]})
    else:
        bytes_launch = None
        if dom == "cg":
            bytes_launch = (CG_BYTES_PER_NODE_ITER * it_mean + CG_BYTES_PER_NODE_SETUP) * N
        elif dom == "node":
            bytes_launch = NODE_BYTES_PER_SWEEP.get(M, 7464) * K * N / max(node_launches_step, 1)
        ach = bytes_launch / (per_launch_ms[dom] * 1e-3) / 1e9 if bytes_launch else None
        roof.update({"bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peaks["hbm_gbs"],
                     "frac": ach / peaks["hbm_gbs"] if ach else None, "peak_source": peaks["source"],
                     "traffic": None})
    if args.precision == "fp64" and M == 4:
        classes = {}
        for cls, (ops, byts) in class_work(solver_kind, K, it_mean, fused=fused).items():
            sec = prof[cls][0] * 1e-3 / args.steps
            if sec <= 0:
                continue
            rate = ops * N / sec
            classes[cls] = {"ms_per_step": sec * 1e3, "fp64_ops_per_node_step": ops,
                            "fp64_issue_frac": rate / FP64_ISSUE_PEAK,
                            "bytes_per_node_step": byts, "gbs": byts * N / sec / 1e9,
                            "hbm_frac": byts * N / sec / 1e9 / peaks["hbm_gbs"]}
        roof["classes"] = classes
        roof["classes_note"] = (
            "fp64_issue_frac: FP64 instructions (DFMA, DADD, DMUL; counted by ncu per node, profiles/) per second "
            "over the FP64 issue peak, 152 SMs x 2 per clock x 2.07 GHz.  On this GPU every class, the diffusion "
            "solve included, is bound by FP64 issue, not HBM: the solve's vectors stay in L2, so its GB/s is "
            "reported against HBM for reference only (the 70%-of-HBM target assumes an HBM-bound stencil).")

    # ---- CPU oracle baseline on one full-size step from the live state (rank 0, N = 1)
    cpu = None
    verr = None
    nxt = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        yh = y[:, :N].cpu().numpy().copy()
        ycopy = y.clone()
        solver.sweep(ycopy, t, dt, M, K)
        g1 = ycopy[:, :N].cpu().numpy()
        m = oracle.Monodomain(wl)
        c0 = time.perf_counter()
        want, _, _, _ = m.step(yh, t, dt, M, K)
        cel = time.perf_counter() - c0
        cpu = {"value": N / cel, "unit": UNIT, "cores": oracle.oracle.threads(), "kind": "oracle",
               "sample": f"one HSDC step of the full {wl.nx}x{wl.ny}x{wl.nz} slab at t={t:.2f} ms"}
        verr = {"V_max_rel_vs_oracle_one_step": float(np.abs(g1[0] - want[0]).max() / np.abs(want[0]).max()),
                "state_max_abs_vs_oracle_one_step": float(np.abs(g1 - want).max())}
        # time-discretisation error over the timed window (oracle, planar strip)
        Va, Vb, osec = _strip_dt8_error(wl, t_w, args.steps, dt)
        Vx = V_end.reshape(wl.nz, wl.ny, wl.nx)
        verr.update({
            "window_ms": [t_w, t_end],
            "discretisation_vs_dt8": _rel(Va, Vb),
            "discretisation_vs_dt8_l2": _rel2(Va, Vb),
            "gpu_slab_vs_oracle_strip_at_window_end": max(_rel(Vx[k, j], Va) for k in (0, wl.nz - 1)
                                                          for j in (0, wl.ny - 1)),
            "gpu_slab_vs_dt8_at_window_end": _rel(Vx[0, 0], Vb),
            "slab_yz_spread": float(np.abs(Vx - Vx[:1, :1, :]).max() / np.abs(Vx).max()),
            "reference": "oracle on the 128x1x1 strip (the slab's planar solution), the window run at dt and "
                         "at dt/8 from the dt run's state at the window start",
            "oracle_seconds": osec})
        if args.precision == "fp64" and not args.no_next_forms:
            nxt = _next_forms(args, wl, y_w, t_w, V_end, Vb, ms_step, solver_kind)
        if args.precision != "fp64":
            ref64 = P.Solver.from_workload(wl, M_max=M)
            y64 = y.clone()
            y64[:, :N] = torch.from_numpy(yh).cuda()
            ref64.sweep(y64, t, dt, M, K)
            g64 = y64[:, :N].cpu().numpy()
            verr["V_max_rel_vs_fp64_gpu_one_step"] = float(np.abs(g1[0] - g64[0]).max() / np.abs(g64[0]).max())
            ref64.close()

    launches = int(sum(v[1] for v in prof.values()))
    if solver_kind == "dct":                 # one profiled "launch" per solve: its kernel passes
        launches += int(prof["cg"][1]) * (DCT_KERNELS_PER_SOLVE(wl) - 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "nodes": N, "n_state": wl.n_state, "M": M, "K": K, "dt_ms": dt,
                   "precision": args.precision, "solver": args.solver,
                   "solve": "DCT-II direct" if solver_kind == "dct" else "iterative",
                   "model": "syn19 (seed 20240530)", "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (state + workspace ~2 GB per GPU)",
                   "window_ms": [t_w, t_end],
                   "untimed_before_window": f"{n_stim} stimulus steps + {args.pre_steps} steps + "
                                            f"{args.warmup} warm-up steps"},
        "s_per_sim_ms": ms_step * 1e-3 / dt,
        "v_error": verr,
        "residual": {"res_inf": res_inf, "y_inf": y_inf},
        "cg_iters_last_step": cg_iters,
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "kernel_launches": {k: v[1] for k, v in prof.items()},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "steps": n_e2e,
                "h2d_bytes_per_step": ns * N * 8, "d2h_bytes_per_step": ns * N * 8},
        "gpu_launches": launches,
        "clocks": clk,
        "next_forms": nxt,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def _next_forms(args, wl, y_w, t_w, V64, Vdt8, ms64, solver_kind):
    """The precision and batching forms beside the headline, on the same box:
    (1) the precision form (FP32 ionic model, FP64 elsewhere) over the same
    window of the same slab from the same state: speedup, its V against the
    FP64 path and both against the dt/8 reference (equal V-error); (2) a small
    ragged batch of HH tissues, batched against one at a time (batches of one,
    identical results)."""
    import numpy as np
    import torch
    import paper_2405_19994_gb300 as P
    from paper_2405_19994_gb300 import inputs as I
    stream = torch.cuda.current_stream()
    M, K, dt, N = wl.M, wl.K, wl.dt, wl.n_nodes
    out = {}
    c0 = time.perf_counter()

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(n):
            fn(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # (1) precision form
    sm = P.Solver.from_workload(wl, M_max=M, precision="mixed", solver=args.solver)
    ym = y_w.clone()
    for k in range(2):                               # warm-up on a copy
        sm.sweep(ym, t_w + k * dt, dt, M, K)
    ym.copy_(y_w)
    tt = [t_w]

    def step_m(k):
        sm.sweep(ym, tt[0], dt, M, K)
        tt[0] += dt
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms_m = timed(step_m, args.steps) / args.steps
    clk = clocks.stop()
    if sm.residual()[0] != 0:
        raise RuntimeError("precision-form step failed")
    Vm = ym[0, :N].cpu().numpy()
    sm.close()
    Vmx = Vm.reshape(wl.nz, wl.ny, wl.nx)
    V64x = V64.reshape(wl.nz, wl.ny, wl.nx)
    out["precision"] = {
        "what": "FP32 ionic model, FP64 state/tables/quadrature/residual, FP64-refined solves",
        "window_ms": [t_w, t_w + args.steps * dt],
        "ms_per_step": ms_m, "fp64_ms_per_step": ms64, "speedup_vs_fp64": ms64 / ms_m,
        "V_max_rel_vs_fp64": _rel(Vm, V64), "V_l2_rel_vs_fp64": _rel2(Vm, V64),
        "V_max_rel_vs_dt8": _rel(Vmx[0, 0], Vdt8), "fp64_V_max_rel_vs_dt8": _rel(V64x[0, 0], Vdt8),
        "clocks": clk}
    # (2) small ragged batch: the first 8 tissues of the 64-tissue batch workload
    wls = I.hh_batch()[:8]
    Mb, Kb, dtb = wls[0].M, wls[0].K, wls[0].dt
    nb_steps = 10
    b = P.Batch.from_workloads(wls, M_max=Mb)
    yb = b.new_state()
    b.init_state(yb, wls[0].V0)
    tb = [0.0]

    def step_b(k):
        b.sweep(yb, tb[0], dtb, Mb, Kb)
        tb[0] += dtb
    for k in range(3):
        step_b(k)
    ms_b = timed(step_b, nb_steps) / nb_steps
    singles = [P.Batch.from_workloads([w], M_max=Mb) for w in wls]
    for s1 in singles:
        s1.set_shape(*b.shape()[:2], 1)
    ys = [s1.new_state() for s1 in singles]
    for s1, y1 in zip(singles, ys):
        s1.init_state(y1, wls[0].V0)
    t1 = [0.0]

    def step_1(k):
        for s1, y1 in zip(singles, ys):
            s1.sweep(y1, t1[0], dtb, Mb, Kb)
        t1[0] += dtb
    for k in range(3):
        step_1(k)
    ms_1 = timed(step_1, nb_steps) / nb_steps
    ok = b.residual()[0] == 0 and all(s1.residual()[0] == 0 for s1 in singles)
    same = all(torch.equal(b.tissue(yb, k), singles[k].tissue(ys[k], 0)) for k in range(len(wls)))
    nodes = int(sum(w.n_nodes for w in wls))
    out["batch"] = {"tissues": len(wls), "nodes": nodes, "steps": nb_steps,
                    "batched_ms_per_step": ms_b, "looped_ms_per_step": ms_1, "speedup": ms_1 / ms_b,
                    "identical_bit_for_bit": bool(same), "ok": bool(ok),
                    "batched_node_updates_per_s": nodes / (ms_b * 1e-3), "graph": bool(b.graph_active())}
    for s1 in singles:
        s1.close()
    b.close()
    out["seconds"] = time.perf_counter() - c0
    return out


def _activation_update(act, v_old, v_new, t_old, dt, level=-40.0):
    """First upward crossing of `level`, linear interpolation between step ends."""
    import torch
    hit = (v_old < level) & (v_new >= level) & torch.isnan(act)
    frac = (level - v_old) / torch.clamp(v_new - v_old, min=1e-300)
    act[hit] = (t_old + frac * dt)[hit]


def _simulate(solver, wl, n_steps, record=True):
    """Run n_steps from rest; per-step CUDA-event timing of the sweeps only.
    Returns (V at the end [N], activation times [N] or None, sweep ms total)."""
    import torch
    N, dt = wl.n_nodes, wl.dt
    y = solver.new_state()
    solver.init_state(y, wl.V0)
    stream = torch.cuda.current_stream()
    act = torch.full((N,), float("nan"), dtype=torch.float64, device=y.device) if record else None
    v_old = y[0, :N].clone() if record else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
    t = 0.0
    for n in range(n_steps):
        ev[n][0].record(stream)
        solver.sweep(y, t, dt, wl.M, wl.K)
        ev[n][1].record(stream)
        if record:
            v_new = y[0, :N]
            _activation_update(act, v_old, v_new, t, dt)
            v_old.copy_(v_new)
        t += dt
    torch.cuda.synchronize()
    rc = solver.residual()[0]
    if rc != 0:
        raise RuntimeError(f"run failed with code {rc}")
    ms = sum(a.elapsed_time(b) for a, b in ev)
    return y[0, :N].clone(), act, ms


def _v_errors(v, ref, act=None, act_ref=None):
    import torch
    out = {"V_max_abs_mV": float((v - ref).abs().max()),
           "V_max_rel": float((v - ref).abs().max() / ref.abs().max()),
           "V_l2_rel": float(torch.linalg.vector_norm(v - ref) / torch.linalg.vector_norm(ref))}
    if act is not None:
        both = ~torch.isnan(act) & ~torch.isnan(act_ref)
        only = torch.isnan(act) ^ torch.isnan(act_ref)
        d = (act - act_ref)[both].abs()
        out.update({"act_max_abs_ms": float(d.max()) if d.numel() else 0.0,
                    "act_mean_abs_ms": float(d.mean()) if d.numel() else 0.0,
                    "activated_nodes": int(both.sum()), "activated_in_one_only": int(only.sum())})
    return out


def run_precision_form(args):
    """The precision form (FP32 ionic model, FP64 state / quadrature / residual,
    refinement CG) on the anisotropic HH slab, against the FP64 path on the
    same GPU over the whole simulated interval, and against the oracle on a
    reduced mesh (the cpu_baseline leg)."""
    import numpy as np
    import torch
    import paper_2405_19994_gb300 as P
    from paper_2405_19994_gb300 import inputs as I

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1 and rank != 0:
        return                                         # single-GPU comparison; replicas add nothing here
    wl = I.hh_aniso_slab()
    if args.nz and args.nz != wl.nz:
        wl = wl.with_mesh(wl.nx, wl.ny, args.nz)
    n_steps = wl.n_steps if args.steps is None else args.steps
    N = wl.n_nodes
    runs = {}
    clocks = ClockSampler(local)
    clocks.start()
    for prec in ("fp64", "mixed"):
        s = P.Solver.from_workload(wl, M_max=wl.M, precision=prec, solver=args.solver)
        _simulate(s, wl, args.warmup, record=False)                 # warm-up (clocks, caches, first launches)
        s.profile(True)
        v, act, ms = _simulate(s, wl, n_steps)
        prof = s.profile_read()
        s.profile(False)
        runs[prec] = {"V": v, "act": act, "ms": ms, "prof": prof, "cg": s.stats(wl.K * wl.M).tolist()}
        s.close()
    clk = clocks.stop()
    r64, rmx = runs["fp64"], runs["mixed"]
    err = _v_errors(rmx["V"], r64["V"], rmx["act"], r64["act"])

    cpu, oracle_err = None, None
    if not args.no_cpu_baseline:
        import oracle
        sub = wl.with_mesh(32, 32, 8)
        m = oracle.Monodomain(sub)
        y = m.init_state()
        act_o = np.full(sub.n_nodes, np.nan)
        t = 0.0
        c0 = time.perf_counter()
        for n in range(sub.n_steps):
            v_old = y[0].copy()
            y, _, _, _ = m.step(y, t, sub.dt, sub.M, sub.K)
            hit = (v_old < -40.0) & (y[0] >= -40.0) & np.isnan(act_o)
            act_o[hit] = t + (-40.0 - v_old[hit]) / (y[0][hit] - v_old[hit]) * sub.dt
            t += sub.dt
        cel = time.perf_counter() - c0
        cpu = {"value": sub.n_nodes * sub.n_steps / cel, "unit": UNIT, "cores": oracle.oracle.threads(),
               "kind": "oracle", "sample": f"the full {sub.n_steps}-step run of the {sub.nx}x{sub.ny}x{sub.nz} "
                                           "reduction of the workload (same physics, fibres and stimulus)"}
        vo = torch.from_numpy(y[0]).cuda()
        ao = torch.from_numpy(act_o).cuda()
        oracle_err = {"mesh": f"{sub.nx}x{sub.ny}x{sub.nz}", "steps": sub.n_steps}
        for prec in ("fp64", "mixed"):
            s = P.Solver.from_workload(sub, M_max=sub.M, precision=prec)
            v, act, _ = _simulate(s, sub, sub.n_steps)
            s.close()
            oracle_err[prec] = _v_errors(v, vo, act, ao)

    launches = int(sum(v[1] for v in rmx["prof"].values()))
    ms_step = rmx["ms"] / n_steps
    line = {
        "metric": METRIC, "value": N * n_steps / (rmx["ms"] * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": n_steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": wl.name, "form": "precision", "nodes": N, "M": wl.M, "K": wl.K, "dt_ms": wl.dt,
                   "solver": args.solver,
                   "T_ms": n_steps * wl.dt, "model": "hh1952", "conductivity": "layered, fibres -60..60 deg",
                   "l2": "inputs larger than L2 (state + workspace ~1.5 GB)"},
        "s_per_sim_ms": ms_step * 1e-3 / wl.dt,
        "fp64": {"value": N * n_steps / (r64["ms"] * 1e-3), "ms_per_step": r64["ms"] / n_steps,
                 "kernels_ms_per_step": {k: v[0] / n_steps for k, v in r64["prof"].items()},
                 "cg_iters_last_step": r64["cg"]},
        "mixed": {"kernels_ms_per_step": {k: v[0] / n_steps for k, v in rmx["prof"].items()},
                  "cg_iters_last_step": rmx["cg"]},
        "speedup_vs_fp64_gpu": r64["ms"] / rmx["ms"],
        "v_error_mixed_vs_fp64_gpu": err,
        "v_error_vs_oracle_reduced_mesh": oracle_err,
        "cpu_baseline": cpu,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_batch_form(args):
    """The batching form: the 64-tissue ragged Hodgkin-Huxley batch stepped by one
    batched launch sequence (recorded CUDA graph, autotuned launch shape) against
    the same tissues stepped one at a time, (a) as batches of one tissue (the
    same kernels: results must be identical bit for bit) and (b) through the
    single-tissue entry point esdc_sweep."""
    import numpy as np
    import torch
    import paper_2405_19994_gb300 as P
    from paper_2405_19994_gb300 import inputs as I

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1 and rank != 0:
        return
    wls = I.hh_batch()
    w0 = wls[0]
    M, K, dt = w0.M, w0.K, w0.dt
    steps = args.steps if args.steps is not None else 20
    nodes = int(sum(w.n_nodes for w in wls))
    stream = torch.cuda.current_stream()

    def timed(step_fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(n):
            step_fn(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # ---- batched
    b = P.Batch.from_workloads(wls, M_max=M, solver=args.solver)
    scratch = b.new_state()
    b.tune(scratch, w0.V0, 0.0, dt, M, K, reps=2)
    shape = b.shape()
    pers = b.persistent()
    del scratch
    yb = b.new_state()
    b.init_state(yb, w0.V0)
    t = [0.0]

    def step_b(k):
        b.sweep(yb, t[0], dt, M, K)
        t[0] += dt
    for k in range(args.warmup):
        step_b(k)
    clocks = ClockSampler(local)
    clocks.start()
    ms_b = timed(step_b, steps)
    clk = clocks.stop()
    rc, res, _ = b.residual()
    if rc != 0:
        raise RuntimeError(f"batched step failed with code {rc}")
    graph = b.graph_active()
    iters = b.stats(K, M)

    # ---- one tissue at a time, as batches of one (same kernels).  They run the
    # launch sequence with the tuned sequence shape whatever mode the tuner chose
    # for the whole batch: a persistent grid over all SMs for one small tissue
    # only adds grid barriers (measured: twice the time).
    singles = [P.Batch.from_workloads([w], M_max=M, solver=args.solver) for w in wls]
    for s1 in singles:
        s1.set_shape(*shape[:2], 1)
    ys = [s1.new_state() for s1 in singles]
    for s1, y1 in zip(singles, ys):
        s1.init_state(y1, w0.V0)
    t1 = [0.0]

    def step_1(k):
        for s1, y1 in zip(singles, ys):
            s1.sweep(y1, t1[0], dt, M, K)
        t1[0] += dt
    for k in range(args.warmup):
        step_1(k)
    ms_1 = timed(step_1, steps)
    for s1 in singles:
        if s1.residual()[0] != 0:
            raise RuntimeError("single-tissue batch failed")
    identical = all(torch.equal(b.tissue(yb, k), singles[k].tissue(ys[k], 0)) for k in range(len(wls)))
    for s1 in singles:
        s1.close()
    del ys

    # ---- the other launch mode on the same batch: one persistent launch per step, or the
    # sequence, whichever the tuner did not pick; the same steps from rest, the same bits
    persist_rows = None
    if args.solver in ("auto", "cheb"):
        persist_rows = []
        modes = [(False, pers[1], pers[2])] if pers[0] else [(True, 512, 128), (True, 512, 512), (True, 256, 128)]
        for mode in modes:
            b.set_persistent(*mode)
            y2 = b.new_state()
            b.init_state(y2, w0.V0)
            t2 = [0.0]

            def step_p(k):
                b.sweep(y2, t2[0], dt, M, K)
                t2[0] += dt
            for k in range(args.warmup):
                step_p(k)
            ms_p = timed(step_p, steps)
            if b.residual()[0] != 0:
                raise RuntimeError("persistent-mode step failed")
            same = all(torch.equal(b.tissue(y2, k), b.tissue(yb, k)) for k in range(len(wls)))
            persist_rows.append({"persistent": mode[0], "threads": mode[1], "node_tile": mode[2],
                                 "ms_per_step": ms_p / steps, "identical_to_tuned": bool(same),
                                 "graph": b.graph_active()})
            del y2
        b.set_persistent(*pers)

    # ---- one tissue at a time through esdc_sweep
    solvers = [P.Solver.from_workload(w, M_max=M, solver=args.solver) for w in wls]
    yv = [s.new_state() for s in solvers]
    for s, y in zip(solvers, yv):
        s.init_state(y, w0.V0)
    t2 = [0.0]

    def step_2(k):
        for s, y in zip(solvers, yv):
            s.sweep(y, t2[0], dt, M, K)
        t2[0] += dt
    for k in range(args.warmup):
        step_2(k)
    ms_2 = timed(step_2, steps)
    maxdiff = 0.0
    for k, (s, y) in enumerate(zip(solvers, yv)):
        if s.residual()[0] != 0:
            raise RuntimeError("single-tissue solver failed")
        ref = b.tissue(yb, k)
        maxdiff = max(maxdiff, float((y[:, :wls[k].n_nodes] - ref).abs().max() / ref.abs().max()))
        s.close()

    # ---- end to end: host state, copies inside the timed region (pinned host buffer)
    yh = torch.empty_like(yb, device="cpu").pin_memory()
    yh.copy_(yb)
    n_e2e = max(1, min(steps, 10))
    torch.cuda.synchronize()
    c0 = time.perf_counter()
    for k in range(n_e2e):
        yb.copy_(yh, non_blocking=True)
        b.sweep(yb, t[0], dt, M, K)
        yh.copy_(yb, non_blocking=True)
        torch.cuda.synchronize()
        t[0] += dt
    e2e_s = time.perf_counter() - c0

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        sample = wls[:4]
        c0 = time.perf_counter()
        done = 0
        for w in sample:
            m = oracle.Monodomain(w)
            y = m.init_state()
            tt = 0.0
            for _ in range(2):
                y, _, _, _ = m.step(y, tt, w.dt, w.M, w.K)
                tt += w.dt
            done += 2 * w.n_nodes
        cel = time.perf_counter() - c0
        cpu = {"value": done / cel, "unit": UNIT, "cores": oracle.oracle.threads(), "kind": "oracle",
               "sample": "2 steps from rest of each of the first 4 tissues of the batch"}
    launches_per_step = 1 + K * (M + 1) + K * M + 1
    # ---- Batch B: P = 16 time slices x M = 3 of one 512 x 512 tissue under Q^par
    qb = run_qpar_batch(args, P, I, torch, timed)
    line = {
        "metric": METRIC, "value": nodes * steps / (ms_b * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_b / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "hh_batch_64 (64 2D HH tissues, sides U[64,512], sigma U[0.05,0.3], seed 4)",
                   "form": "batch", "tissues": len(wls), "nodes": nodes, "M": M, "K": K, "dt_ms": dt,
                   "solver": args.solver,
                   "l2": "inputs larger than L2 (batch state and workspace ~3.7 GB)"},
        "s_per_sim_ms": ms_b / steps * 1e-3 / dt,
        "launch_shape": {"node_waves": shape[0], "cg_threads": shape[1], "cg_blocks": shape[2],
                         "persistent": pers[0], "persistent_threads": pers[1], "node_tile": pers[2]},
        "other_launch_modes": persist_rows,
        "graph": graph,
        "graph_error": b.graph_error() or None,
        "looped_batches_of_one": {"value": nodes * steps / (ms_1 * 1e-3), "ms_per_step": ms_1 / steps,
                                  "identical_to_batched": bool(identical)},
        "looped_single_solver": {"value": nodes * steps / (ms_2 * 1e-3), "ms_per_step": ms_2 / steps,
                                 "max_rel_diff_vs_batched": maxdiff},
        "speedup_vs_looped_batches_of_one": ms_1 / ms_b,
        "speedup_vs_looped_single_solver": ms_2 / ms_b,
        "cg_iters_last_step_max": int(iters.max()),
        "residual_max": float(res.max()),
        "cpu_baseline": cpu,
        "e2e": {"value": nodes * n_e2e / e2e_s, "unit": UNIT, "steps": n_e2e,
                "h2d_bytes_per_step": int(yb.numel() * 8), "d2h_bytes_per_step": int(yb.numel() * 8)},
        "gpu_launches": launches_per_step * steps,
        "clocks": clk,
        "qpar_batch_b": qb,
    }
    b.close()
    print(json.dumps(line), flush=True)


def run_qpar_batch(args, P, I, torch, timed):
    """Batch B: one 2D 512 x 512 Hodgkin-Huxley tissue (h = 0.25 mm, corner
    stimulus), P = 16 consecutive steps as time slices, M = 3, 4 Q^par
    iterations per solve (eq. def_Q), batched against looping the slices one at a
    time (same kernels: identical results)."""
    w = I.hh_sheet_32().with_mesh(512, 512, 1, name="hh_sheet_512")
    Pn, M, iters, dt = 16, w.M, 4, w.dt
    reps = 5
    b = P.Batch.from_workloads([w] * Pn, M_max=M, solver=args.solver)
    yin, yout = b.new_state(), b.new_state()
    y0 = b.new_state()
    b.init_state(y0, w.V0)

    def solve_b(k):
        yin.copy_(y0)
        b.qpar(yin, yout, 0.0, dt, M, iters)
    for k in range(max(2, args.warmup)):
        solve_b(k)
    ms_b = timed(solve_b, reps)
    if b.residual()[0] != 0:
        raise RuntimeError("Q^par batch failed")
    graph = b.graph_active()
    singles = [P.Batch.from_workloads([w], M_max=M, solver=args.solver) for _ in range(Pn)]
    yi = [s.new_state() for s in singles]
    yo = [s.new_state() for s in singles]
    y0s = b.tissue(y0, 0).clone()

    def solve_1(k):
        ends = None
        for it in range(iters):
            for p, s in enumerate(singles):
                s.tissue(yi[p], 0).copy_(y0s if (p == 0 or ends is None) else ends[p - 1])
                s.sweep_from(yi[p], yo[p], p * dt, dt, M, 1, from_iterate=it > 0)
            ends = [s.tissue(yo[p], 0) for p, s in enumerate(singles)]
            ends = [e.clone() for e in ends]
    for k in range(max(2, args.warmup)):
        solve_1(k)
    ms_1 = timed(solve_1, reps)
    identical = all(torch.equal(b.tissue(yout, p), singles[p].tissue(yo[p], 0)) for p in range(Pn))
    for s in singles:
        s.close()
    b.close()
    nodes = Pn * w.n_nodes
    return {"workload": "hh_sheet_512 (512x512 HH, corner stimulus), P=16 slices x M=3, 4 Q^par iterations",
            "ms_per_solve": ms_b / reps, "node_updates_per_s": nodes / (ms_b / reps * 1e-3),
            "slice_sweeps_per_s": Pn * iters / (ms_b / reps * 1e-3), "graph": graph,
            "looped_slices": {"ms_per_solve": ms_1 / reps, "identical_to_batched": bool(identical)},
            "speedup_vs_looped_slices": ms_1 / ms_b}


def run_adjoint_form(args):
    """The differentiation form: 2D 256 x 256 HH tissue with a log-normal
    conductivity field, M = 3, K = 4, dt = 0.025 ms, T = 20 ms (800 steps), loss
    = half the squared misfit of V at 64 seeded sensor nodes after every step
    against a seeded target run (another field, g_Na x 1.05, g_K x 0.95).
    Times the forward run (with one checkpoint per step) and the adjoint
    (recomputation + reverse sweeps), and checks the gradient along a seeded
    direction of the field against central differences of the forward map."""
    import numpy as np
    import torch
    import paper_2405_19994_gb300 as P
    from paper_2405_19994_gb300 import inputs as I

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1 and rank != 0:
        return
    n = args.nz if args.nz else 256                       # side length (the flag is reused for this 2D form)
    wl = I.hh_field_sheet(n)
    nsteps = args.steps if args.steps is not None else wl.n_steps
    rng = np.random.default_rng(5)
    sens_h = np.sort(rng.choice(wl.n_nodes, size=64, replace=False)).astype(np.int32)
    sens = torch.from_numpy(sens_h).cuda()
    s = P.Solver.from_workload(wl, M_max=wl.M)
    y0 = s.new_state()
    s.init_state(y0, wl.V0)
    tr = torch.empty((nsteps, 64), dtype=torch.float64, device="cuda")
    ck = torch.empty((nsteps, s.n_state, s.ld), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def forward(sig, params):
        s.set_params(params)
        s.set_conductivity_field(sig)
        y = y0.clone()
        s.adjoint_forward(y, 0.0, wl.dt, wl.M, wl.K, nsteps, sens, tr, ck)
        torch.cuda.synchronize()
        if s.residual()[0] != 0:
            raise RuntimeError("forward run failed")
        return tr.clone()

    p_t = wl.params.copy()
    p_t[0] *= 1.05
    p_t[1] *= 0.95
    target = forward(I.lognormal_field(n, n, 1, seed=55), p_t)
    forward(wl.sigma_field, wl.params)                     # warm-up
    clocks = ClockSampler(local)
    clocks.start()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(stream)
    trs = forward(wl.sigma_field, wl.params)
    e[1].record(stream)
    dtr = (trs - target).contiguous()
    gsig, gpar, _ = s.adjoint_backward(ck, 0.0, wl.dt, wl.M, wl.K, nsteps, sens, dtr)
    e[2].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_f, ms_b = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    loss = 0.5 * float((dtr ** 2).sum())

    # gradient check along a seeded direction of the field (central differences, eps = 1e-6)
    eps = 1e-6
    d = wl.sigma_field * np.random.default_rng(7).normal(size=wl.n_nodes)
    Lp = 0.5 * float(((forward(wl.sigma_field + eps * d, wl.params) - target) ** 2).sum())
    Lm = 0.5 * float(((forward(wl.sigma_field - eps * d, wl.params) - target) ** 2).sum())
    fd = (Lp - Lm) / (2 * eps)
    ad = float(gsig.cpu().numpy() @ d)

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        sub = I.hh_field_sheet(32)
        m = oracle.Monodomain(sub, cg_tol=1e-15)
        y = m.init_state()
        t = 0.0
        c0 = time.perf_counter()
        for _ in range(80):
            y, _, _, _ = m.step(y, t, sub.dt, sub.M, sub.K)
            t += sub.dt
        cel = time.perf_counter() - c0
        cpu = {"value": sub.n_nodes * 80 / cel, "unit": UNIT, "cores": oracle.oracle.threads(), "kind": "oracle",
               "sample": "80 forward steps of the 32x32 field sheet (the oracle has no adjoint; forward only)"}
    nodes = wl.n_nodes
    line = {
        "metric": METRIC, "value": nodes * nsteps / ((ms_f + ms_b) * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": nsteps, "warmup": 1, "ms_per_step": (ms_f + ms_b) / nsteps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"hh_field_sheet_{n} (log-normal sigma field, seed 5)", "form": "adjoint",
                   "nodes": nodes, "M": wl.M, "K": wl.K, "dt_ms": wl.dt, "T_ms": nsteps * wl.dt, "sensors": 64,
                   "value_is": "node-updates/s of forward + backward together"},
        "forward_ms": ms_f, "backward_ms": ms_b, "backward_over_forward": ms_b / ms_f,
        "forward_node_updates_per_s": nodes * nsteps / (ms_f * 1e-3),
        "loss": loss, "dL_dgNa": float(gpar[0]), "dL_dgK": float(gpar[1]),
        "grad_check_field": {"adjoint": ad, "central_difference": fd,
                             "rel_err": abs(ad - fd) / abs(fd) if fd != 0.0 else None,
                             "abs_err": abs(ad - fd), "eps": eps},
        "checkpoint_bytes": int(ck.numel() * 8),
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_fas_form(args):
    """Algorithm HSDC with two levels (M = 3, 2) against single-level Q^par
    (M = 3) on P = 16 consecutive steps of the 512 x 512 HH sheet (corner
    stimulus, dt = 0.025 ms): the error of the last slice's end value against
    the sequential collocation solution after each iteration, and the time per
    iteration, both on the GPU."""
    import numpy as np
    import torch
    import paper_2405_19994_gb300 as P
    from paper_2405_19994_gb300 import inputs as I

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1 and rank != 0:
        return
    n = args.nz if args.nz else 512
    w = I.hh_sheet_32().with_mesh(n, n, 1, name=f"hh_sheet_{n}")
    Pn, M1, M2, dt = 16, 3, 2, w.dt
    iters = args.steps if args.steps is not None else 10
    stream = torch.cuda.current_stream()
    # state at t0 = 0.4 ms: inside the stimulus window, the upstroke under way
    one = P.Batch.from_workloads([w], M_max=M1, solver=args.solver)
    y0 = one.new_state()
    one.init_state(y0, w.V0)
    t0 = 0.0
    for _ in range(16):
        one.sweep(y0, t0, dt, M1, w.K)
        t0 += dt
    # sequential collocation reference: P steps with 40 sweeps each
    yref = y0.clone()
    t = t0
    for _ in range(Pn):
        one.sweep(yref, t, dt, M1, 40)
        t += dt
    if one.residual()[0] != 0:
        raise RuntimeError("reference run failed")
    ref = yref[0, :w.n_nodes].clone()

    fine = P.Batch.from_workloads([w] * Pn, M_max=M1, solver=args.solver)
    coarse = [P.Batch.from_workloads([w], M_max=M2, solver=args.solver) for _ in range(Pn)]
    yin, yout = fine.new_state(), fine.new_state()
    last = int(fine.offsets[Pn - 1])

    def err():
        v = yout[0, last:last + w.n_nodes]
        return float((v - ref).abs().max() / ref.abs().max())

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def load():
        yin.zero_()
        fine.tissue(yin, 0).copy_(y0[:, :w.n_nodes])

    # three levels, M = 3, 2, 1: a second Q^par level of the same slices, Q^seq at M = 1
    M3 = 1
    mid = P.Batch.from_workloads([w] * Pn, M_max=M2, solver=args.solver)
    coarse3 = [P.Batch.from_workloads([w], M_max=M3, solver=args.solver) for _ in range(Pn)]

    out = {"hsdc2": [], "hsdc3": [], "qpar": []}
    clocks = ClockSampler(local)
    clocks.start()
    for k in range(1, iters + 1):
        load()
        ms = timed(lambda: P.esdc.hsdc2(fine, coarse, yin, yout, t0, dt, M1, M2, k))
        out["hsdc2"].append({"iters": k, "ms": ms, "err": err()})
        load()
        ms = timed(lambda: P.esdc.hsdc([fine, mid], coarse3, yin, yout, t0, dt, (M1, M2, M3), k))
        out["hsdc3"].append({"iters": k, "ms": ms, "err": err()})
        load()
        ms = timed(lambda: fine.qpar(yin, yout, t0, dt, M1, k))
        if fine.residual()[0] != 0:
            raise RuntimeError("Q^par failed")
        out["qpar"].append({"iters": k, "ms": ms, "err": err()})
    # Q^par needs up to P iterations to carry y0 across all slices: extend it
    for k in (Pn, Pn + 4, Pn + 8, Pn + 12):
        load()
        ms = timed(lambda: fine.qpar(yin, yout, t0, dt, M1, k))
        out["qpar"].append({"iters": k, "ms": ms, "err": err()})

    clk = clocks.stop()

    def first_below(rows, tol):
        for r in rows:
            if r["err"] < tol:
                return r
        return None
    tol = 1e-8
    h, q = first_below(out["hsdc2"], tol), first_below(out["qpar"], tol)
    h6, q6 = first_below(out["hsdc2"], 1e-6), first_below(out["qpar"], 1e-6)
    h3, h36 = first_below(out["hsdc3"], tol), first_below(out["hsdc3"], 1e-6)
    nodes = Pn * w.n_nodes
    line = {
        "metric": METRIC, "value": (nodes / (h["ms"] * 1e-3)) if h else None, "unit": UNIT, "n_gpus": 1,
        "steps": Pn, "warmup": 0, "ms_per_step": (h["ms"] / Pn) if h else None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"hh_sheet_{n} (corner stimulus), P=16 slices from t0={t0:.2f} ms",
                   "form": "fas", "levels": [M1, M2], "dt_ms": dt, "solver": args.solver,
                   "value_is": "node-updates/s of the two-level solve to 1e-8 relative error of the last slice"},
        "tolerance": tol,
        "hsdc2_to_tol": h, "qpar_to_tol": q,
        "speedup_hsdc2_vs_qpar_to_tol": (q["ms"] / h["ms"]) if (h and q) else None,
        "hsdc2_to_1e-6": h6, "qpar_to_1e-6": q6,
        "speedup_hsdc2_vs_qpar_to_1e-6": (q6["ms"] / h6["ms"]) if (h6 and q6) else None,
        "hsdc3_levels": [M1, M2, M3], "hsdc3_to_tol": h3, "hsdc3_to_1e-6": h36,
        "history": out,
        "clocks": clk,
    }
    for c in coarse + coarse3:
        c.close()
    mid.close()
    fine.close()
    print(json.dumps(line), flush=True)


def run_peaks_form(args):
    """The FMA throughput ceilings the FP64 kernels are compared with: the
    library's probe (independent FMA chains on every SM) in FP64 and FP32,
    best of a few launches after a warm-up, with the SM clocks sampled."""
    import torch
    import paper_2405_19994_gb300 as P

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1 and rank != 0:
        return
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    out = {}
    for name, fp32, n in (("fp64", False, 40000), ("fp32", True, 2000000)):
        P.esdc.fma_probe(fp32, n // 10, stream)                       # warm-up
        best = None
        for _ in range(max(args.warmup, 3)):
            ms, flops = P.esdc.fma_probe(fp32, n, stream)
            tf = flops / (ms * 1e-3) / 1e12
            best = tf if best is None else max(best, tf)
        out[name] = best
    clk = clocks.stop()
    sm = clk.get("sm_mhz") or 2070.0
    line = {"metric": "FMA throughput ceiling", "value": out["fp64"], "unit": "TFLOP/s", "n_gpus": 1,
            "fp64_tflops": out["fp64"], "fp32_tflops": out["fp32"],
            "fp64_fma_per_sm_per_clk": out["fp64"] * 1e12 / 2 / (152 * sm * 1e6),
            "fp64_derived_peak_tflops": FP64_PEAK_TFLOPS, "clocks": clk,
            "config": {"form": "peaks", "probe": "esdc_fma_probe: 4 x 256 threads per SM, 8 FMA chains each"}}
    print(json.dumps(line), flush=True)


def run_sheet_form(args):
    """Config 1: the 32x32 HH parity sheet (corner stimulus, M = 3, K = 4,
    dt = 0.025 ms, T = 4 ms, 160 steps) on the GPU, its V error at T against
    the oracle, and the oracle's own time for the whole run on this host's
    cores (OMP_NUM_THREADS sets how many)."""
    import numpy as np
    import torch
    import paper_2405_19994_gb300 as P
    from paper_2405_19994_gb300 import inputs as I

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1 and rank != 0:
        return
    wl = I.hh_sheet_32()
    n = wl.n_steps
    s = P.Solver.from_workload(wl)
    stream = torch.cuda.current_stream()

    def run():
        y = s.new_state()
        s.init_state(y, wl.V0)
        t = 0.0
        for _ in range(n):
            s.sweep(y, t, wl.dt, wl.M, wl.K)
            t += wl.dt
        return y
    for _ in range(max(1, args.warmup)):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    y = run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if s.residual()[0] != 0:
        raise RuntimeError("run failed")
    got = y[0, :wl.n_nodes].cpu().numpy()
    cpu, verr = None, None
    if not args.no_cpu_baseline:
        import oracle
        m = oracle.Monodomain(wl)
        yo = m.init_state()
        t = 0.0
        c0 = time.perf_counter()
        for _ in range(n):
            yo, _, _, _ = m.step(yo, t, wl.dt, wl.M, wl.K)
            t += wl.dt
        cel = time.perf_counter() - c0
        cpu = {"value": wl.n_nodes * n / cel, "unit": UNIT, "cores": oracle.oracle.threads(), "kind": "oracle",
               "sample": "the whole 160-step run", "s_per_sim_ms": cel / wl.T}
        verr = float(np.abs(got - yo[0]).max() / np.abs(yo[0]).max())
    line = {
        "metric": METRIC, "value": wl.n_nodes * n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": n,
        "warmup": max(1, args.warmup), "ms_per_step": ms / n, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "form": "sheet", "nodes": wl.n_nodes, "M": wl.M, "K": wl.K, "dt_ms": wl.dt,
                   "T_ms": wl.T, "l2": "latency-bound parity case (1024 nodes, L2-resident)"},
        "s_per_sim_ms": ms * 1e-3 / wl.T,
        "V_max_rel_vs_oracle_at_T": verr,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 40; the precision form runs its whole interval)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-next-forms", action="store_true",
                    help="headline: skip the precision-form and batch comparisons beside the timed window")
    ap.add_argument("--pre-steps", type=int, default=100,
                    help="headline: untimed steps after the stimulus before the warm-up and the timed window")
    ap.add_argument("--nz", type=int, default=None, help="slab depth (default: the workload's own)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="mixed: the precision form (FP32 ionic model, FP64 elsewhere)")
    ap.add_argument("--solver", choices=["auto", "cg", "dct", "cheb"], default="auto",
                    help="diffusion solves (headline, precision, batch and fas forms): auto (the DCT-II direct solve "
                         "for the scalar sigma on the FP64 path where its transforms are cheap, else as cheb), cheb (Chebyshev semi-iteration on a "
                         "known spectral interval, else CG), cg (Jacobi-PCG) or dct (the DCT-II direct solve; "
                         "headline form only)")
    ap.add_argument("--form", choices=["plain", "precision", "batch", "adjoint", "fas", "sheet", "peaks"],
                    default="plain",
                    help="precision: FP64 vs mixed on the anisotropic HH slab (256x256x64, T = 10 ms); "
                         "batch: the 64-tissue ragged HH batch against looped single-tissue steps; "
                         "adjoint: forward + discrete adjoint on the 256x256 HH conductivity-field sheet; "
                         "fas: two-level Algorithm HSDC against Q^par on 16 slices of the 512x512 HH sheet; "
                         "sheet: the 32x32 HH parity sheet's full run against the oracle; "
                         "peaks: the FP64/FP32 FMA throughput ceilings")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.solver == "dct" and (args.form != "plain" or args.impl != "ours"):     # DCT: scalar sigma, FP64
        ap.error("--solver dct applies to the headline form only")
    if args.steps is None and args.form == "plain":
        args.steps = 40
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "precision":
        run_precision_form(args)
    elif args.form == "batch":
        run_batch_form(args)
    elif args.form == "adjoint":
        run_adjoint_form(args)
    elif args.form == "fas":
        run_fas_form(args)
    elif args.form == "sheet":
        run_sheet_form(args)
    elif args.form == "peaks":
        run_peaks_form(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
