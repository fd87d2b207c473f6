"""Seeded synthetic inputs: ionic-model parameter sets, workload descriptions
and random states.

This module is the only code that the CUDA path and the CPU oracle share.  It
holds none of the method's arithmetic: parameter sets are published constants
or seeded draws, and states are seeded random numbers in physical ranges.

Workloads (the paper measures on none of its own data; Sec. 5 uses square
domains with uniform meshes and self-excited or stimulated waves):

* ``hh_sheet_32``: 2D 32x32 cells, h = 0.25 mm, Hodgkin-Huxley 1952, rest
  V = -75 mV, 0.5 uA/mm^2 for [0, 1) ms on the 4x4 corner, M = 3, K = 4,
  dt = 0.025 ms, T = 4 ms.
* ``syn19_slab``: 3D 128x128x32 cells (524,288 nodes), h = 0.2 mm, the seeded
  19-state synthetic stiff model, planar stimulus 0.5 uA/mm^2 for [0, 1) ms on
  the two cell layers at x = 0, M = 4, K = 6, dt = 0.05 ms, T = 50 ms.

Both use sigma = 0.17 mS/mm, chi = 140 /mm, C_m = 0.01 uF/mm^2 (Sec. 5 gives
chi and C_m; sigma_i = 0.17 is used as the conductivity).
"""
from __future__ import annotations

import dataclasses
import numpy as np

MODEL_HH1952 = 0
MODEL_SYN19 = 1

N_STATE = {MODEL_HH1952: 4, MODEL_SYN19: 19}
N_GATE = {MODEL_HH1952: 3, MODEL_SYN19: 12}
N_PARAM = {MODEL_HH1952: 7, MODEL_SYN19: 88}

SYN19_SEED = 20240530


def hh1952_params(v_rest: float = -75.0) -> np.ndarray:
    """Hodgkin & Huxley (1952) constants: [gNa, gK, gL, ENa, EK, EL, Vrest].

    Conductances 120, 36, 0.3 mS/cm^2 = 1.2, 0.36, 0.003 mS/mm^2; reversal
    potentials +115, -12, +10.613 mV relative to rest."""
    return np.array([1.2, 0.36, 0.003, v_rest + 115.0, v_rest - 12.0, v_rest + 10.613, v_rest],
                    dtype=np.float64)


def syn19_params(seed: int = SYN19_SEED) -> np.ndarray:
    """Seeded parameters of the 19-state synthetic stiff model (88 values).

    Layout: 12 gates x (Vh [mV], k [mV], r [1/ms], ln rho, Vr [mV], sr [mV]),
    then [G_f, E_f, G_s, E_s, G_K, E_K, G_K1, G_b, E_b, c_K6], then tau_1..6 [ms].
    Gate rates r * rho^s lie in [1e2, 1e4] /ms: the base rates are stratified
    log-uniformly over [1e2, 6e3] (one stratum per gate, in random order) and
    rho is uniform in [1.1, 1.6]."""
    rng = np.random.default_rng(seed)
    strata = rng.permutation(12)
    # (Vh range, k range) per gate role
    roles = ([((-60.0, -50.0), (4.0, 6.0))] * 3 +        # g1..g3 fast activation
             [((-45.0, -35.0), (4.0, 6.0))] * 2 +        # g4, g5 plateau activation
             [((-68.0, -62.0), (4.0, 6.0))] +            # g6 depolarisation sensor
             [((-65.0, -55.0), (-8.0, -6.0))] * 2 +      # g7, g8 inward rectifier
             [((-70.0, -30.0), (5.0, 10.0)), ((-70.0, -30.0), (-10.0, -5.0))] * 2)
    p = []
    for q, (vh, kk) in enumerate(roles):
        u = rng.uniform(0.0, 1.0)
        r = float(np.exp(np.log(1e2) + (strata[q] + u) / 12.0 * np.log(60.0)))
        p += [rng.uniform(*vh), rng.uniform(*kk), r, float(np.log(rng.uniform(1.1, 1.6))),
              rng.uniform(-70.0, -30.0), rng.uniform(5.0, 15.0)]
    p += [0.06, 40.0, 0.006, 40.0, 0.02, -85.0, 0.012, 0.0015, -60.0, 0.5]
    p += [3.0, 15.0, 20.0, 5.0, 10.0, 20.0]
    return np.asarray(p, dtype=np.float64)


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    h: float
    model: int
    params: np.ndarray
    V0: float
    M: int
    K: int
    dt: float
    T: float
    sigma: float = 0.17
    chi: float = 140.0
    Cm: float = 0.01
    # layered anisotropic conductivity: {"sxx","syy","sxy","szz"} -> [nz] arrays, or None
    layers: dict | None = None
    # heterogeneous isotropic conductivity: one value per node [N] (mS/mm), or None
    sigma_field: np.ndarray | None = None
    # order of the Laplacian: 2 (3/5/7-point) or 4 (five-point fourth-order differences per axis)
    order: int = 2
    # stimulus boxes: [x0, x1, y0, y1, z0, z1] node index ranges (half-open)
    boxes: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 6), np.int32))
    amp: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    t_on: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    t_off: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_state(self) -> int:
        return N_STATE[self.model]

    @property
    def n_gate(self) -> int:
        return N_GATE[self.model]

    @property
    def n_steps(self) -> int:
        return int(round(self.T / self.dt))

    def with_mesh(self, nx: int, ny: int, nz: int, name: str | None = None) -> "Workload":
        """Same physics on another mesh; stimulus boxes are clipped to it."""
        b = self.boxes.copy()
        b[:, 1] = np.minimum(b[:, 1], nx)
        b[:, 3] = np.minimum(b[:, 3], ny)
        b[:, 5] = np.minimum(b[:, 5], nz)
        dim = 1 if (ny == 1 and nz == 1) else (2 if nz == 1 else 3)
        layers = self.layers
        if layers is not None and nz != self.nz:     # same fibre rotation over the new depth
            sl = float(np.max(layers["sxx"] + layers["syy"] - layers["szz"]))
            layers = fibre_layers(nz, sigma_l=sl, sigma_t=float(layers["szz"][0]))
        field = self.sigma_field
        if field is not None and (nx, ny, nz) != (self.nx, self.ny, self.nz):
            field = None                                # a per-node field does not carry over
        return dataclasses.replace(self, name=name or f"{self.name}@{nx}x{ny}x{nz}",
                                   nx=nx, ny=ny, nz=nz, dim=dim, boxes=b, layers=layers, sigma_field=field)


def fibre_layers(nz: int, sigma_l: float = 0.17, sigma_t: float = 0.02,
                 theta0_deg: float = -60.0, theta1_deg: float = 60.0) -> dict:
    """Conductivity tensor of fibres lying in the xy-plane whose angle rotates
    linearly through the depth, theta(z) from theta0 (bottom layer) to theta1
    (top layer): sigma = sigma_t I + (sigma_l - sigma_t) f f^T, f = (cos, sin, 0)."""
    th = np.deg2rad(np.linspace(theta0_deg, theta1_deg, nz)) if nz > 1 else np.array([np.deg2rad(theta0_deg)])
    d = sigma_l - sigma_t
    return {"sxx": sigma_t + d * np.cos(th) ** 2, "syy": sigma_t + d * np.sin(th) ** 2,
            "sxy": d * np.sin(th) * np.cos(th), "szz": np.full(nz, sigma_t)}


def hh_sheet_32() -> Workload:
    return Workload(name="hh_sheet_32x32", dim=2, nx=32, ny=32, nz=1, h=0.25,
                    model=MODEL_HH1952, params=hh1952_params(), V0=-75.0,
                    M=3, K=4, dt=0.025, T=4.0,
                    boxes=np.array([[0, 4, 0, 4, 0, 1]], np.int32),
                    amp=np.array([0.5]), t_on=np.array([0.0]), t_off=np.array([1.0]))


def syn19_slab() -> Workload:
    return Workload(name="syn19_slab_128x128x32", dim=3, nx=128, ny=128, nz=32, h=0.2,
                    model=MODEL_SYN19, params=syn19_params(), V0=-83.4,
                    M=4, K=6, dt=0.05, T=50.0,
                    boxes=np.array([[0, 2, 0, 128, 0, 32]], np.int32),
                    amp=np.array([0.5]), t_on=np.array([0.0]), t_off=np.array([1.0]))


def hh_aniso_slab() -> Workload:
    """The precision-form workload: 3D 256x256x64 (4,194,304 nodes), h = 0.2 mm,
    Hodgkin-Huxley, fibres rotating from -60 to +60 degrees through the depth
    (sigma_l = 0.17, sigma_t = 0.02 mS/mm), planar stimulus on the two cell
    layers at x = 0 for [0, 1) ms, M = 4, K = 6, dt = 0.05 ms, T = 10 ms."""
    return Workload(name="hh_aniso_slab_256x256x64", dim=3, nx=256, ny=256, nz=64, h=0.2,
                    model=MODEL_HH1952, params=hh1952_params(), V0=-75.0,
                    M=4, K=6, dt=0.05, T=10.0, layers=fibre_layers(64),
                    boxes=np.array([[0, 2, 0, 256, 0, 64]], np.int32),
                    amp=np.array([0.5]), t_on=np.array([0.0]), t_off=np.array([1.0]))


def random_state(wl: Workload, seed: int, ld: int | None = None) -> np.ndarray:
    """A seeded mid-wave-like state [n_state, ld] (columns >= n_nodes are 0).

    V: a smooth front along x between -85 and +30 mV plus small noise;
    auxiliaries uniform in [0, 1]; gates uniform in [0, 1]."""
    rng = np.random.default_rng(seed)
    N = wl.n_nodes
    ld = N if ld is None else ld
    y = np.zeros((wl.n_state, ld), np.float64)
    ix = np.arange(N) % wl.nx
    x0 = rng.uniform(0.3, 0.7) * wl.nx
    width = max(1.0, 0.05 * wl.nx)
    y[0, :N] = -85.0 + 115.0 / (1.0 + np.exp((ix - x0) / width)) + rng.normal(0.0, 0.5, N)
    y[1:, :N] = rng.uniform(0.0, 1.0, (wl.n_state - 1, N))
    return y


def hh_batch(n: int = 64, seed: int = 4, side: tuple = (64, 512), sigma: tuple = (0.05, 0.3),
             patch: int = 8) -> list:
    """The ragged batch of the batching form: n seeded 2D Hodgkin-Huxley tissues,
    each side length drawn uniformly from side[0]..side[1] (nx and ny
    independently), sigma uniformly from sigma[0]..sigma[1] mS/mm, and a
    patch x patch stimulus (0.5 uA/mm^2 for [0, 1) ms) at a uniformly drawn
    position.  h = 0.25 mm, rest -75 mV, M = 3, K = 4, dt = 0.025 ms, T = 4 ms."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx, ny = (int(v) for v in rng.integers(side[0], side[1] + 1, size=2))
        sg = float(rng.uniform(*sigma))
        px, py = min(patch, nx), min(patch, ny)
        x0 = int(rng.integers(0, nx - px + 1))
        y0 = int(rng.integers(0, ny - py + 1))
        out.append(Workload(name=f"hh_batch[{k}]_{nx}x{ny}", dim=2 if ny > 1 else 1, nx=nx, ny=ny, nz=1, h=0.25,
                            model=MODEL_HH1952, params=hh1952_params(), V0=-75.0, M=3, K=4, dt=0.025, T=4.0,
                            sigma=sg, boxes=np.array([[x0, x0 + px, y0, y0 + py, 0, 1]], np.int32),
                            amp=np.array([0.5]), t_on=np.array([0.0]), t_off=np.array([1.0])))
    return out


def lognormal_field(nx: int, ny: int, nz: int = 1, seed: int = 5, sigma0: float = 0.17, amp: float = 0.3,
                    corr: float = 8.0) -> np.ndarray:
    """A smooth log-normal conductivity field sigma0 exp(amp g) [nz*ny*nx],
    g a seeded Gaussian random field of unit variance with Gaussian covariance
    of correlation length `corr` nodes (white noise filtered in Fourier space)."""
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(nz, ny, nx))
    k = [np.fft.fftfreq(n) for n in (nz, ny, nx)]
    kz, ky, kx = np.meshgrid(*k, indexing="ij")
    filt = np.exp(-0.5 * (2 * np.pi * corr) ** 2 * (kx ** 2 + ky ** 2 + (kz ** 2 if nz > 1 else 0.0)) / 2)
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    g = (g - g.mean()) / max(g.std(), 1e-300)
    return (sigma0 * np.exp(amp * g)).reshape(-1)


def hh_field_sheet(n: int = 256, seed: int = 5) -> Workload:
    """The differentiation-form tissue: 2D n x n, h = 0.25 mm, Hodgkin-Huxley,
    conductivity 0.17 exp(0.3 g) mS/mm with g a smooth seeded Gaussian field,
    corner stimulus (4x4 nodes, 0.5 uA/mm^2, [0, 1) ms), M = 3, K = 4,
    dt = 0.025 ms, T = 20 ms."""
    return Workload(name=f"hh_field_sheet_{n}", dim=2, nx=n, ny=n, nz=1, h=0.25,
                    model=MODEL_HH1952, params=hh1952_params(), V0=-75.0, M=3, K=4, dt=0.025, T=20.0,
                    sigma_field=lognormal_field(n, n, 1, seed=seed),
                    boxes=np.array([[0, 4, 0, 4, 0, 1]], np.int32),
                    amp=np.array([0.5]), t_on=np.array([0.0]), t_off=np.array([1.0]))
