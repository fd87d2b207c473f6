"""ctypes view of the C oracle in this directory (test infrastructure only).

Every function mirrors one C entry point of ``esdc_oracle.h``; see the C
sources for the passages of the paper each one follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["orc_colloc.c", "orc_model.c", "orc_space.c", "orc_sweep.c"]
LIB_PATH = os.path.join(_HERE, "liborc.so")

SOLVE_DCT, SOLVE_CG, SOLVE_DENSE = 0, 1, 2
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64: no fast-math, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "esdc_oracle.h")]
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("ctx", C.c_void_p), ("f_I", C.c_void_p), ("solve_I", C.c_void_p),
                ("f_E", C.c_void_p), ("lam_yinf", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("sweeps_done", C.c_int), ("res_inf", C.c_double), ("y_inf", C.c_double),
                ("solve_fail", C.c_int)]


class _Mono(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.c_double), ("sigma", C.c_double), ("chi", C.c_double), ("Cm", C.c_double),
                ("model", C.c_int), ("mp", C.c_void_p), ("n_mp", C.c_int),
                ("nbox", C.c_int), ("box", C.c_void_p), ("amp", C.c_void_p),
                ("t_on", C.c_void_p), ("t_off", C.c_void_p),
                ("solver", C.c_int), ("cg_tol", C.c_double), ("cg_maxit", C.c_int),
                ("ionic_off", C.c_int), ("lay_sxx", C.c_void_p), ("lay_syy", C.c_void_p),
                ("lay_sxy", C.c_void_p), ("lay_szz", C.c_void_p), ("sig_node", C.c_void_p),
                ("order", C.c_int), ("work", C.c_void_p)]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        L.orc_radau_nodes.argtypes = [C.c_int, _D]
        L.orc_gauss_legendre.argtypes = [C.c_int, _D, _D]
        L.orc_collocation_q.argtypes = [C.c_int, _D, _D]
        L.orc_fornberg_weights.argtypes = [C.c_int, _D, _D]
        L.orc_phi.argtypes = [C.c_double, C.c_int, _D]
        L.orc_aij.argtypes = [C.c_int, _D, _D, C.c_double, _D]
        L.orc_hsdc_step.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_double, C.c_int,
                                    C.c_double, C.c_double, _D, _D, _D, _D, C.POINTER(_Stats)]
        L.orc_hsdc_step_from.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_double, C.c_int,
                                         C.c_double, C.c_double, _D, _D, _D, _D, _D, C.POINTER(_Stats)]
        L.orc_hsdc_step_tau.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int, C.c_double, C.c_int,
                                        C.c_double, C.c_double, _D, _D, _D, _D, _D, _D, C.POINTER(_Stats)]
        L.orc_mono_problem.argtypes = [C.POINTER(_Mono), C.POINTER(_Problem)]
        L.orc_mono_free.argtypes = [C.POINTER(_Mono)]
        L.orc_mono_init.argtypes = [C.POINTER(_Mono), C.c_double, _D]
        L.orc_ionic_point.argtypes = [C.c_int, _D, _D, _D, _D, _D]
        L.orc_ionic_rest.argtypes = [C.c_int, _D, C.c_double, _D]
        L.orc_laplacian.argtypes = [C.POINTER(_Mono), _D, _D]
        L.orc_solve_shifted.argtypes = [C.POINTER(_Mono), C.c_int, C.c_double, _D, _D]
        L.orc_conductivity.argtypes = [C.POINTER(_Mono), _D, _D]
        L.orc_solve_A.argtypes = [C.POINTER(_Mono), C.c_int, C.c_double, _D, _D]
        L.orc_stability_R1.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                       C.c_double, C.c_int]
        L.orc_stability_R1.restype = C.c_double
        L.orc_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def lagrange_matrix(nodes: np.ndarray, points: np.ndarray) -> np.ndarray:
    """L[i, j] = l_j(points[i]), l_j the Lagrange basis through `nodes` (the
    interpolator I_l of Sec. 3.2, product form)."""
    nodes = np.asarray(nodes, np.float64)
    L = np.ones((len(points), len(nodes)))
    for i, x in enumerate(points):
        for j, cj in enumerate(nodes):
            for k, ck in enumerate(nodes):
                if k != j:
                    L[i, j] *= (x - ck) / (cj - ck)
    return L


def radau_nodes(M: int) -> np.ndarray:
    c = np.zeros(M + 1)
    if lib().orc_radau_nodes(M, _p(c)):
        raise ValueError("bad M")
    return c


def gauss_legendre(n: int):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_legendre(n, _p(x), _p(w))
    return x, w


def collocation_q(M: int) -> np.ndarray:
    c = radau_nodes(M)
    q = np.zeros(M * M)
    lib().orc_collocation_q(M, _p(c), _p(q))
    return q.reshape(M, M)


def fornberg_weights(M: int, c: np.ndarray | None = None) -> np.ndarray:
    """w[k, l] = weight of p(c_{l+1}) in p^{(k)}(0), k = 0..M-1."""
    c = radau_nodes(M) if c is None else np.ascontiguousarray(c, np.float64)
    w = np.zeros(M * M)
    lib().orc_fornberg_weights(M, _p(c), _p(w))
    return w.reshape(M, M)


def phi(z: float, kmax: int) -> np.ndarray:
    out = np.zeros(kmax)
    lib().orc_phi(float(z), kmax, _p(out))
    return out


def aij(M: int, z: float) -> np.ndarray:
    c = radau_nodes(M)
    w = fornberg_weights(M, c).ravel().copy()
    a = np.zeros(M * M)
    lib().orc_aij(M, _p(c), _p(w), float(z), _p(a))
    return a.reshape(M, M)


def ionic_point(model: int, params: np.ndarray, u: np.ndarray):
    ns = len(u)
    u = np.ascontiguousarray(u, np.float64)
    params = np.ascontiguousarray(params, np.float64)
    fE, lam, yinf = np.zeros(ns), np.zeros(ns), np.zeros(ns)
    lib().orc_ionic_point(model, _p(params), _p(u), _p(fE), _p(lam), _p(yinf))
    return fE, lam, yinf


def ionic_rest(model: int, params: np.ndarray, V0: float) -> np.ndarray:
    ns = 4 if model == 0 else 19
    u = np.zeros(ns)
    lib().orc_ionic_rest(model, _p(np.ascontiguousarray(params, np.float64)), float(V0), _p(u))
    return u


def threads() -> int:
    """OpenMP threads the oracle's loops run on."""
    return int(lib().orc_threads())


def stability_R1(lI: float, lE: float, le: float, M: int, K: int, tol: float = 0.0,
                 plain_sdc: bool = False) -> float:
    return lib().orc_stability_R1(lI, lE, le, M, K, tol, int(plain_sdc))


class Monodomain:
    """A monodomain problem (mesh, conductivity, ionic model, stimulus) in the oracle.

    ``wl`` is an ``inputs.Workload``; ``solver`` selects the oracle's linear
    solve (DCT-II by default, the paper's solver)."""

    def __init__(self, wl, solver: int = SOLVE_DCT, cg_tol: float = 1e-15, cg_maxit: int = 2000,
                 ionic_off: bool = False):
        self.wl = wl
        self._keep = [np.ascontiguousarray(wl.params, np.float64),
                      np.ascontiguousarray(wl.boxes, np.int32),
                      np.ascontiguousarray(wl.amp, np.float64),
                      np.ascontiguousarray(wl.t_on, np.float64),
                      np.ascontiguousarray(wl.t_off, np.float64)]
        mp, box, amp, ton, toff = self._keep
        lay = [None] * 4
        layers = getattr(wl, "layers", None)
        if layers is not None:
            lay_arrs = [np.ascontiguousarray(layers[k], np.float64) for k in ("sxx", "syy", "sxy", "szz")]
            assert all(len(a) == wl.nz for a in lay_arrs)
            self._keep += lay_arrs
            lay = [a.ctypes.data for a in lay_arrs]
            if solver == SOLVE_DCT:
                solver = SOLVE_CG        # DCT-II does not diagonalise the layered operator
        field = getattr(wl, "sigma_field", None)
        fptr = None
        if field is not None:
            f = np.ascontiguousarray(field, np.float64).reshape(-1)
            assert len(f) == wl.n_nodes and layers is None
            self._keep.append(f)
            fptr = f.ctypes.data
            if solver == SOLVE_DCT:
                solver = SOLVE_CG        # nor a heterogeneous one
        self.m = _Mono(wl.dim, wl.nx, wl.ny, wl.nz, wl.h, wl.sigma, wl.chi, wl.Cm, wl.model,
                       mp.ctypes.data, len(mp), len(amp), box.ctypes.data, amp.ctypes.data,
                       ton.ctypes.data, toff.ctypes.data, solver, cg_tol, cg_maxit, int(ionic_off),
                       lay[0], lay[1], lay[2], lay[3], fptr, int(getattr(wl, "order", 2)), None)
        self.P = _Problem()
        if lib().orc_mono_problem(C.byref(self.m), C.byref(self.P)):
            raise ValueError("invalid monodomain description")
        self.N = wl.n_nodes
        self.ns = wl.n_state

    def __del__(self):
        try:
            lib().orc_mono_free(C.byref(self.m))
        except Exception:
            pass

    def init_state(self, V0: float | None = None) -> np.ndarray:
        y = np.zeros(self.ns * self.N)
        lib().orc_mono_init(C.byref(self.m), float(self.wl.V0 if V0 is None else V0), _p(y))
        return y.reshape(self.ns, self.N)

    def laplacian(self, v: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(v, np.float64)
        out = np.zeros(self.N)
        lib().orc_laplacian(C.byref(self.m), _p(v), _p(out))
        return out

    def conductivity(self, v: np.ndarray) -> np.ndarray:
        """A v with A = div(sigma grad) (conductivity included)."""
        v = np.ascontiguousarray(v, np.float64)
        out = np.zeros(self.N)
        lib().orc_conductivity(C.byref(self.m), _p(v), _p(out))
        return out

    def solve_A(self, g: float, b: np.ndarray, x0: np.ndarray | None = None,
                method: int | None = None) -> np.ndarray:
        """Solve (I - g A) x = b."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.N) if x0 is None else np.array(x0, np.float64)
        rc = lib().orc_solve_A(C.byref(self.m), self.m.solver if method is None else method,
                               float(g), _p(b), _p(x))
        if rc:
            raise RuntimeError(f"oracle solve failed ({rc})")
        return x

    def solve_shifted(self, g: float, b: np.ndarray, x0: np.ndarray | None = None,
                      method: int | None = None) -> np.ndarray:
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.N) if x0 is None else np.array(x0, np.float64)
        rc = lib().orc_solve_shifted(C.byref(self.m), self.m.solver if method is None else method,
                                     float(g), _p(b), _p(x))
        if rc:
            raise RuntimeError(f"oracle solve failed ({rc})")
        return x

    def step(self, y_n: np.ndarray, t_n: float, dt: float, M: int, K: int, tol: float = 0.0,
             plain_sdc: bool = False, want_colloc: bool = False, want_resid: bool = False,
             colloc_in: np.ndarray | None = None, tau: np.ndarray | None = None):
        """One HSDC step; returns (y_next[ns, N], stats dict, colloc, resid).

        colloc_in [M, ns, N] (optional) starts the sweeps from that iterate
        instead of y^0 = 1 (x) y_n (orc_hsdc_step_from); tau [M, ns, N]
        (optional) is the FAS correction added to the right-hand side
        (orc_hsdc_step_tau).  K = 0 returns the residual at the given iterate."""
        y_n = np.ascontiguousarray(y_n, np.float64).reshape(-1)
        n = len(y_n)
        y1 = np.zeros(n)
        col = np.zeros(M * n) if want_colloc else None
        res = np.zeros(M * n) if want_resid else None
        cin = None if colloc_in is None else np.ascontiguousarray(colloc_in, np.float64).reshape(-1)
        if cin is not None and len(cin) != M * n:
            raise ValueError("colloc_in must hold M x n_state x N values")
        tv = None if tau is None else np.ascontiguousarray(tau, np.float64).reshape(-1)
        if tv is not None and len(tv) != M * n:
            raise ValueError("tau must hold M x n_state x N values")
        st = _Stats()
        rc = lib().orc_hsdc_step_tau(C.byref(self.P), M, K, tol, int(plain_sdc), float(t_n), float(dt),
                                     _p(y_n), _p(cin) if cin is not None else None,
                                     _p(tv) if tv is not None else None, _p(y1),
                                     _p(col) if col is not None else None,
                                     _p(res) if res is not None else None, C.byref(st))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")
        stats = dict(sweeps=st.sweeps_done, res_inf=st.res_inf, y_inf=st.y_inf)
        shp = (self.ns, self.N)
        return (y1.reshape(shp), stats,
                None if col is None else col.reshape((M,) + shp),
                None if res is None else res.reshape((M,) + shp))

    def qpar(self, y0: np.ndarray, t0: float, dt: float, P: int, M: int, iters: int):
        """Q^par iteration (eq. prec_picard_seq with Q = Q^par, eq. def_Q) for P
        consecutive steps from y0 at t0, started from z^0 = 1 (x) y0 in every
        slice (the paper's Burn-in is not specified).  Iteration k+1: every
        slice p runs one sweep from its iterate z_p^k with y_{p,0} = y0 (p = 0)
        or the last node y_{p-1,M}^k of the previous slice's iterate.
        Returns the iterates [P, M, ns, N] after `iters` iterations."""
        y0 = np.asarray(y0, np.float64).reshape(self.ns, self.N)
        Z = np.broadcast_to(y0, (P, M, self.ns, self.N)).copy()
        for _ in range(iters):
            ends = Z[:, M - 1].copy()
            newZ = np.empty_like(Z)
            for p in range(P):
                yn = y0 if p == 0 else ends[p - 1]
                _, _, col, _ = self.step(yn, t0 + p * dt, dt, M, 1, want_colloc=True, colloc_in=Z[p])
                newZ[p] = col
            Z = newZ
        return Z

    def hsdc2(self, y0: np.ndarray, t0: float, dt: float, P: int, M1: int, M2: int, iters: int,
              Z0: np.ndarray | None = None):
        """Algorithm HSDC (Sec. 3.2) with two levels, M = M1, M2 (M1 > M2 Radau
        nodes), over P consecutive steps from y0 at t0, without Burn-in (not
        specified: z^0 = 1 (x) y0 in every slice).  One iteration:
          tau = D_2(S z) - S D_1(z), per slice S R_1(z_p) - R_2(S z_p), with
                R = b - D the collocation residual vectors (the slice couplings
                cancel, and row 0 of tau vanishes because c_M = 1 on both levels);
          coarse: one Q^seq sweep from S z with tau: slice p starts from the
                new end value of slice p-1;
          fine:   one Q^par sweep from z + T(z_2 - S z): slice p starts from the
                corrected end value of slice p-1 of that iterate.
        S interpolates the fine node values at the coarse nodes, T the coarse
        ones at the fine nodes (Lagrange through c_1..c_M).  Z0 [P, M1, ns, N]
        (optional) replaces z^0, with row 0 of slice p the end of slice p-1.
        Returns the fine iterates [P, M1, ns, N]."""
        y0 = np.asarray(y0, np.float64).reshape(self.ns, self.N)
        R = lagrange_matrix(radau_nodes(M1)[1:], radau_nodes(M2)[1:])       # [M2, M1]
        T = lagrange_matrix(radau_nodes(M2)[1:], radau_nodes(M1)[1:])       # [M1, M2]
        Z = np.broadcast_to(y0, (P, M1, self.ns, self.N)).copy() if Z0 is None else np.array(Z0, np.float64)
        Y0 = np.broadcast_to(y0, (P, self.ns, self.N)).copy()              # row 0 of every slice
        if Z0 is not None:
            Y0[1:] = Z[:-1, M1 - 1]
        for _ in range(iters):
            SZ = np.einsum("ij,pjsn->pisn", R, Z)
            tau = np.empty((P, M2, self.ns, self.N))
            for p in range(P):
                _, _, _, r1 = self.step(Y0[p], t0 + p * dt, dt, M1, 0, want_resid=True, colloc_in=Z[p])
                _, _, _, r2 = self.step(Y0[p], t0 + p * dt, dt, M2, 0, want_resid=True, colloc_in=SZ[p])
                tau[p] = np.einsum("ij,jsn->isn", R, r1) - r2
            Z2 = np.empty_like(SZ)
            for p in range(P):                                             # Q^seq on the coarse level
                yi = y0 if p == 0 else Z2[p - 1, M2 - 1]
                _, _, Z2[p], _ = self.step(yi, t0 + p * dt, dt, M2, 1, want_colloc=True, colloc_in=SZ[p],
                                           tau=tau[p])
            W = Z + np.einsum("ij,pjsn->pisn", T, Z2 - SZ)                 # coarse-grid correction
            Znew = np.empty_like(Z)
            for p in range(P):                                             # Q^par on the fine level
                Y0[p] = y0 if p == 0 else W[p - 1, M1 - 1]
                _, _, Znew[p], _ = self.step(Y0[p], t0 + p * dt, dt, M1, 1, want_colloc=True, colloc_in=W[p])
            Z = Znew
        return Z

    def hsdc(self, y0: np.ndarray, t0: float, dt: float, P: int, Ms, iters: int,
             Z0: np.ndarray | None = None):
        """Algorithm HSDC (Sec. 3.2) with L = len(Ms) >= 2 levels of M_1 > ... > M_L
        Radau nodes over P consecutive steps from y0 at t0, without Burn-in
        (z^0 = 1 (x) y0 in every slice).  S_l restricts level l to level l+1 and
        T_l prolongs back: Lagrange interpolation through the nodes c_1..c_M of
        the source level (row 0, the slice's initial value, is kept).  With
        R_l(z; tau) = b + tau - D_l(z) the residual vectors, one iteration is
          level 1:      z_1^{k+1/2} = z_1^k, tau_1 = 0;
          l = 2..L:     tau_l = S R_{l-1}(z_{l-1}^{k+1/2}; tau_{l-1}) - R_l(S z_{l-1}^{k+1/2}; 0)
                        (that is D_l(S z) - S D_{l-1}(z) + S tau_{l-1});
                        for l < L one Q^par sweep from S z_{l-1}^{k+1/2} with tau_l gives z_l^{k+1/2};
          level L:      one Q^seq sweep from S z_{L-1}^{k+1/2} with tau_L gives z_L^{k+1};
          l = L-1..1:   one Q^par sweep from z_l^{k+1/2} + T (z_{l+1}^{k+1} - S z_l^{k+1/2})
                        with tau_l gives z_l^{k+1}.
        A Q^par sweep starts slice p from the end value of slice p-1 of the
        iterate it sweeps (y0 for slice 0), the Q^seq sweep from the new end
        value of slice p-1; a residual of slice p uses the initial value its
        iterate was swept with.  Z0 [P, M_1, ns, N] (optional) replaces z^0.
        Returns the level-1 iterates [P, M_1, ns, N].  With two levels this is
        hsdc2."""
        Ms = [int(M) for M in Ms]
        L = len(Ms)
        if L < 2 or any(Ms[l + 1] >= Ms[l] for l in range(L - 1)):
            raise ValueError("need L >= 2 levels with M_1 > M_2 > ... > M_L")
        y0 = np.asarray(y0, np.float64).reshape(self.ns, self.N)
        nodes = [radau_nodes(M)[1:] for M in Ms]
        Smat = [lagrange_matrix(nodes[l], nodes[l + 1]) for l in range(L - 1)]    # [M_{l+1}, M_l]
        Tmat = [lagrange_matrix(nodes[l + 1], nodes[l]) for l in range(L - 1)]    # [M_l, M_{l+1}]

        def restrict(l, X):                      # level l -> l + 1 (0-based levels)
            return np.einsum("ij,pjsn->pisn", Smat[l], X)

        def prolong(l, X):                       # level l + 1 -> l
            return np.einsum("ij,pjsn->pisn", Tmat[l], X)

        def residuals(l, Z, Y0, tau):
            out = np.empty_like(Z)
            for p in range(P):
                _, _, _, out[p] = self.step(Y0[p], t0 + p * dt, dt, Ms[l], 0, want_resid=True, colloc_in=Z[p],
                                            tau=None if tau is None else tau[p])
            return out

        def sweep_par(l, Zs, tau):
            Zn = np.empty_like(Zs)
            Y0 = np.empty((P, self.ns, self.N))
            for p in range(P):
                Y0[p] = y0 if p == 0 else Zs[p - 1, Ms[l] - 1]
                _, _, Zn[p], _ = self.step(Y0[p], t0 + p * dt, dt, Ms[l], 1, want_colloc=True, colloc_in=Zs[p],
                                           tau=None if tau is None else tau[p])
            return Zn, Y0

        Z1 = np.broadcast_to(y0, (P, Ms[0], self.ns, self.N)).copy() if Z0 is None else np.array(Z0, np.float64)
        Y01 = np.broadcast_to(y0, (P, self.ns, self.N)).copy()
        if Z0 is not None:
            Y01[1:] = Z1[:-1, Ms[0] - 1]
        for _ in range(iters):
            Zh, Y0h, SZ, tau = [Z1], [Y01], [None], [None]
            for l in range(1, L):                                           # down to the coarsest level
                SZ.append(restrict(l - 1, Zh[l - 1]))
                tau.append(restrict(l - 1, residuals(l - 1, Zh[l - 1], Y0h[l - 1], tau[l - 1]))
                           - residuals(l, SZ[l], Y0h[l - 1], None))
                if l < L - 1:
                    zl, yl = sweep_par(l, SZ[l], tau[l])
                    Zh.append(zl)
                    Y0h.append(yl)
            Zc = np.empty_like(SZ[L - 1])                                   # Q^seq on the coarsest level
            for p in range(P):
                yi = y0 if p == 0 else Zc[p - 1, Ms[L - 1] - 1]
                _, _, Zc[p], _ = self.step(yi, t0 + p * dt, dt, Ms[L - 1], 1, want_colloc=True,
                                           colloc_in=SZ[L - 1][p], tau=tau[L - 1][p])
            Znew = Zc
            for l in range(L - 2, -1, -1):                                  # back up, correcting each level
                Znew, Y0new = sweep_par(l, Zh[l] + prolong(l, Znew - SZ[l + 1]), tau[l])
            Z1, Y01 = Znew, Y0new
        return Z1

    def run(self, y0: np.ndarray, t0: float, dt: float, nsteps: int, M: int, K: int):
        y = np.array(y0, np.float64)
        t = t0
        for _ in range(nsteps):
            y, _, _, _ = self.step(y, t, dt, M, K)
            t += dt
        return y
