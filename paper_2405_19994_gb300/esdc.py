"""Python binding of the HSDC C library (include/esdc.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``libesdc.so``.  Torch supplies device memory and streams; tensors are passed to
the library as raw pointers (``data_ptr()``) together with the current CUDA
stream.  The binding fails loudly when the library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libesdc.so")

ESDC_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "CG_NOT_CONVERGED", -4: "NONFINITE",
          -5: "DEVICE_TIMEOUT", -6: "UNSUPPORTED", -7: "NO_MEMORY", -8: "TOO_LARGE"}
MODEL_HH1952, MODEL_SYN19 = 0, 1


class EsdcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"esdc error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class esdc_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double)]


class esdc_options(C.Structure):
    _fields_ = [("M_max", C.c_int), ("tol_cg", C.c_double), ("cg_maxit", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("solver", C.c_int), ("fuse_node1", C.c_int)]


_lib = None
_VP, _D, _I64 = C.c_void_p, C.c_double, C.c_int64


def lib() -> C.CDLL:
    """Load libesdc.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        sig = {
            "esdc_default_options": (None, [C.POINTER(esdc_options)]),
            "esdc_create": (C.c_int, [C.POINTER(esdc_mesh), _D, _D, _D, C.c_int, C.POINTER(_D), C.c_int,
                                      C.POINTER(esdc_options), C.POINTER(_VP)]),
            "esdc_destroy": (None, [_VP]),
            "esdc_last_error": (C.c_char_p, [_VP]),
            "esdc_set_stimulus": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int), C.POINTER(_D), C.POINTER(_D),
                                            C.POINTER(_D)]),
            "esdc_state_size": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(_I64), C.POINTER(_I64)]),
            "esdc_set_conductivity_layers": (C.c_int, [_VP, C.POINTER(_D), C.POINTER(_D), C.POINTER(_D),
                                                       C.POINTER(_D)]),
            "esdc_set_conductivity_field": (C.c_int, [_VP, C.POINTER(_D)]),
            "esdc_set_stencil_order": (C.c_int, [_VP, C.c_int]),
            "esdc_get_solver": (C.c_int, [_VP, C.POINTER(C.c_int)]),
            "esdc_table_errors": (C.c_int, [C.c_int, C.POINTER(_D), C.c_int, C.c_int, _D, C.POINTER(_D)]),
            "esdc_init_state": (C.c_int, [_VP, _VP, _D, _VP]),
            "esdc_sweep": (C.c_int, [_VP, _VP, _D, _D, C.c_int, C.c_int, _VP]),
            "esdc_sweep_host": (C.c_int, [_VP, _VP, _I64, _D, _D, C.c_int, C.c_int, _VP]),
            "esdc_residual": (C.c_int, [_VP, C.POINTER(_D), C.POINTER(_D), C.POINTER(_D)]),
            "esdc_stats": (C.c_int, [_VP, C.POINTER(C.c_int), C.c_int]),
            "esdc_keep_residual": (C.c_int, [_VP, C.c_int]),
            "esdc_profile": (C.c_int, [_VP, C.c_int]),
            "esdc_profile_read": (C.c_int, [_VP, C.POINTER(_D), C.POINTER(C.c_longlong)]),
            "esdc_collocation": (C.c_int, [_VP, _VP, _VP, _VP]),
            "esdc_coefficients": (C.c_int, [_VP, _VP, _I64, C.c_int, _VP, _VP]),
            "esdc_diffusion_solve": (C.c_int, [_VP, _D, _VP, _VP, C.POINTER(C.c_int), _VP]),
            "esdc_ionic": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
            "esdc_math_check": (C.c_int, [_VP, _I64, _VP, _VP, _VP]),
            "esdc_fma_probe": (C.c_int, [C.c_int, _I64, C.POINTER(_D), C.POINTER(_D), _VP]),
            "esdc_diffusion_solve_static": (C.c_int, [C.POINTER(esdc_mesh), _D, _VP, _VP, _D, C.c_int, C.c_int,
                                                      C.POINTER(C.c_int), _VP]),
            "esdc_set_params": (C.c_int, [_VP, C.POINTER(_D), C.c_int]),
            "esdc_debug_barrier": (C.c_int, [_VP, C.c_int, C.c_uint]),
            "esdc_adjoint_forward": (C.c_int, [_VP, _VP, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP,
                                               _VP]),
            "esdc_adjoint_backward": (C.c_int, [_VP, _VP, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP,
                                                _VP, _VP, C.POINTER(_D), _VP]),
            "esdc_batch_create": (C.c_int, [C.c_int, C.POINTER(esdc_mesh), C.POINTER(_D), _D, _D, C.c_int,
                                            C.POINTER(_D), C.c_int, C.POINTER(esdc_options), C.POINTER(_VP)]),
            "esdc_batch_destroy": (None, [_VP]),
            "esdc_batch_last_error": (C.c_char_p, [_VP]),
            "esdc_batch_set_stimulus": (C.c_int, [_VP, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(_D),
                                                  C.POINTER(_D), C.POINTER(_D)]),
            "esdc_batch_layout": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(_I64), C.POINTER(_I64)]),
            "esdc_batch_init_state": (C.c_int, [_VP, _VP, _D, _VP]),
            "esdc_batch_sweep": (C.c_int, [_VP, _VP, C.POINTER(_D), _D, C.c_int, C.c_int, _VP]),
            "esdc_batch_residual": (C.c_int, [_VP, C.POINTER(_D), C.POINTER(_D)]),
            "esdc_batch_sweep_from": (C.c_int, [_VP, _VP, _VP, C.POINTER(_D), _D, C.c_int, C.c_int, C.c_int, _VP]),
            "esdc_batch_qpar": (C.c_int, [_VP, _VP, _VP, _D, _D, C.c_int, C.c_int, _VP]),
            "esdc_batch_sweep_ex": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(_D), _D, C.c_int, C.c_int, C.c_int, C.c_int,
                                              _VP]),
            "esdc_batch_iterate": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_VP)]),
            "esdc_interp": (C.c_int, [_VP, C.c_int, _I64, _VP, C.c_int, _I64, C.c_int, _I64, C.POINTER(_D), _D, _VP]),
            "esdc_hsdc2": (C.c_int, [_VP, C.POINTER(_VP), _VP, _VP, _D, _D, C.c_int, C.c_int, C.c_int, _VP]),
            "esdc_hsdc": (C.c_int, [C.POINTER(_VP), C.POINTER(_VP), C.POINTER(C.c_int), C.c_int, _VP, _VP, _D, _D,
                                    C.c_int, _VP]),
            "esdc_batch_stats": (C.c_int, [_VP, C.POINTER(C.c_int), C.c_int]),
            "esdc_batch_set_graph": (C.c_int, [_VP, C.c_int]),
            "esdc_batch_graph_active": (C.c_int, [_VP]),
            "esdc_batch_graph_error": (C.c_char_p, [_VP]),
            "esdc_batch_set_shape": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
            "esdc_batch_set_persistent": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
            "esdc_batch_get_persistent": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "esdc_batch_get_shape": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "esdc_batch_tune": (C.c_int, [_VP, _VP, _D, _D, _D, C.c_int, C.c_int, C.c_int, _VP]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _stream(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t) -> int:
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return t.data_ptr()


def fma_probe(fp32: bool, n: int, stream=None):
    """FMA throughput of the device (esdc_fma_probe): returns (ms, flops)."""
    ms, fl = C.c_double(), C.c_double()
    rc = lib().esdc_fma_probe(int(fp32), n, C.byref(ms), C.byref(fl), _stream(stream))
    if rc != ESDC_OK:
        raise EsdcError(rc, "esdc_fma_probe failed")
    return ms.value, fl.value


def math_check(x, stream=None):
    """The library's FP64 exp and reciprocal of a float64 CUDA tensor x."""
    import torch
    ex, rc = torch.empty_like(x), torch.empty_like(x)
    rc_ = lib().esdc_math_check(_ptr(x), x.numel(), _ptr(ex), _ptr(rc), _stream(stream))
    if rc_ != ESDC_OK:
        raise EsdcError(rc_, "esdc_math_check failed")
    return ex, rc


class Solver:
    """One HSDC solver handle: a mesh, conductivity and ionic model on the current GPU.

    Every method maps onto one C entry point of the same name without the
    ``esdc_`` prefix."""

    def __init__(self, dim: int, nx: int, ny: int, nz: int, h: float, sigma: float, chi: float,
                 Cm: float, model: int, params, M_max: int = 8, tol_cg: float = 1e-14,
                 cg_maxit: int = 200, precond: bool = True, precision: str = "fp64", solver: str = "auto",
                 fuse_node1: bool = True):
        self._h = None
        L = lib()
        mesh = esdc_mesh(dim, nx, ny, nz, h)
        opt = esdc_options()
        L.esdc_default_options(C.byref(opt))
        opt.M_max, opt.tol_cg, opt.cg_maxit, opt.precond = M_max, tol_cg, cg_maxit, int(precond)
        if precision not in ("fp64", "mixed"):
            raise ValueError("precision must be 'fp64' or 'mixed'")
        opt.precision = 1 if precision == "mixed" else 0
        if solver not in ("auto", "cg", "dct", "cheb"):
            raise ValueError("solver must be 'auto', 'cg', 'dct' or 'cheb'")
        opt.solver = {"auto": 0, "cg": 1, "dct": 2, "cheb": 3}[solver]
        opt.fuse_node1 = int(bool(fuse_node1))
        p = np.ascontiguousarray(params, np.float64)
        out = _VP()
        rc = L.esdc_create(C.byref(mesh), sigma, chi, Cm, model, p.ctypes.data_as(C.POINTER(_D)), len(p),
                           C.byref(opt), C.byref(out))
        if rc != ESDC_OK:
            raise EsdcError(rc, "esdc_create failed")
        self._h = out.value
        ns, nn, ld = C.c_int(), _I64(), _I64()
        self._check(L.esdc_state_size(self._h, C.byref(ns), C.byref(nn), C.byref(ld)))
        self.n_state, self.n_nodes, self.ld = ns.value, nn.value, ld.value
        self.M_max = M_max
        self.params = p.copy()

    @classmethod
    def from_workload(cls, wl, **kw) -> "Solver":
        s = cls(wl.dim, wl.nx, wl.ny, wl.nz, wl.h, wl.sigma, wl.chi, wl.Cm, wl.model, wl.params, **kw)
        s.set_stimulus(wl.boxes, wl.amp, wl.t_on, wl.t_off)
        if getattr(wl, "layers", None) is not None:
            s.set_conductivity_layers(wl.layers)
        if getattr(wl, "sigma_field", None) is not None:
            s.set_conductivity_field(wl.sigma_field)
        if getattr(wl, "order", 2) != 2:
            s.set_stencil_order(wl.order)
        return s

    def _check(self, rc: int):
        if rc != ESDC_OK:
            msg = lib().esdc_last_error(self._h).decode() if self._h else ""
            raise EsdcError(rc, msg)

    def close(self):
        if self._h:
            lib().esdc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- ABI calls
    def set_stimulus(self, boxes, amp, t_on, t_off):
        b = np.ascontiguousarray(boxes, np.int32).reshape(-1)
        a, on, off = (np.ascontiguousarray(x, np.float64) for x in (amp, t_on, t_off))
        n = len(a)
        self._check(lib().esdc_set_stimulus(self._h, n, b.ctypes.data_as(C.POINTER(C.c_int)),
                                            a.ctypes.data_as(C.POINTER(_D)), on.ctypes.data_as(C.POINTER(_D)),
                                            off.ctypes.data_as(C.POINTER(_D))))

    def set_conductivity_layers(self, layers):
        """layers: {"sxx","syy","sxy","szz"} -> arrays of length nz, or None for the scalar sigma."""
        if layers is None:
            self._check(lib().esdc_set_conductivity_layers(self._h, None, None, None, None))
            return
        arrs = [np.ascontiguousarray(layers[k], np.float64) for k in ("sxx", "syy", "sxy", "szz")]
        self._check(lib().esdc_set_conductivity_layers(self._h, *[a.ctypes.data_as(C.POINTER(_D)) for a in arrs]))

    def set_stencil_order(self, order: int):
        """2: the 3/5/7-point Laplacian; 4: the fourth-order five-point differences per axis."""
        self._check(lib().esdc_set_stencil_order(self._h, int(order)))

    def solver_in_use(self) -> str:
        """The diffusion solver the solves take now: "dct", "cheb" or "cg"."""
        v = C.c_int(0)
        self._check(lib().esdc_get_solver(self._h, C.byref(v)))
        return {1: "cg", 2: "dct", 3: "cheb"}[v.value]

    def set_conductivity_field(self, sigma):
        """Per-node conductivity [N] (mS/mm), or None for the scalar sigma."""
        if sigma is None:
            self._check(lib().esdc_set_conductivity_field(self._h, None))
            return
        f = np.ascontiguousarray(sigma, np.float64).reshape(-1)
        if len(f) != self.n_nodes:
            raise ValueError("the field needs one value per mesh node")
        self._check(lib().esdc_set_conductivity_field(self._h, f.ctypes.data_as(C.POINTER(_D))))

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float64)
        self._check(lib().esdc_set_params(self._h, p.ctypes.data_as(C.POINTER(_D)), len(p)))
        self.params = p.copy()

    def adjoint_forward(self, y, t0: float, dt: float, M: int, K: int, nsteps: int, sens, traces, ckpt, stream=None):
        """esdc_adjoint_forward: y in/out, traces [nsteps, nsens], ckpt [nsteps, n_state, ld]."""
        import torch
        assert sens.dtype == torch.int32 and sens.is_cuda and sens.is_contiguous()
        self._check(lib().esdc_adjoint_forward(self._h, _ptr(y), t0, dt, M, K, nsteps, sens.numel(), sens.data_ptr(),
                                               _ptr(traces) if sens.numel() else None, _ptr(ckpt), _stream(stream)))

    def adjoint_backward(self, ckpt, t0: float, dt: float, M: int, K: int, nsteps: int, sens, dtraces,
                         dy_final=None, want_y0: bool = False, stream=None):
        """esdc_adjoint_backward: returns (dL/dsigma [N], dL/d(g_Na, g_K) [2], dL/dy0 or None)."""
        import torch
        gsig = torch.zeros(self.n_nodes, dtype=torch.float64, device="cuda")
        gy0 = torch.zeros((self.n_state, self.ld), dtype=torch.float64, device="cuda") if want_y0 else None
        gpar = np.zeros(2)
        self._check(lib().esdc_adjoint_backward(
            self._h, _ptr(ckpt), t0, dt, M, K, nsteps, sens.numel(), sens.data_ptr(),
            _ptr(dtraces) if sens.numel() else None, _ptr(dy_final) if dy_final is not None else None,
            _ptr(gy0) if gy0 is not None else None, _ptr(gsig), gpar.ctypes.data_as(C.POINTER(_D)),
            _stream(stream)))
        return gsig, gpar, gy0

    def new_state(self, device=None):
        import torch
        return torch.zeros((self.n_state, self.ld), dtype=torch.float64, device=device or "cuda")

    def init_state(self, y, V0: float, stream=None):
        self._check(lib().esdc_init_state(self._h, _ptr(y), V0, _stream(stream)))
        return y

    def sweep(self, y, t: float, dt: float, M: int, K: int, stream=None):
        self._check(lib().esdc_sweep(self._h, _ptr(y), t, dt, M, K, _stream(stream)))
        return y

    def sweep_host(self, y_host: np.ndarray, t: float, dt: float, M: int, K: int, stream=None):
        """y_host: host float64 array [n_state, ld_host] (C-contiguous, e.g. pinned)."""
        if isinstance(y_host, np.ndarray):
            assert y_host.dtype == np.float64 and y_host.flags.c_contiguous
            ptr, ld = y_host.ctypes.data, y_host.shape[1]
        else:   # a CPU torch tensor (pinned memory for asynchronous copies)
            assert y_host.dtype.is_floating_point and y_host.is_contiguous() and not y_host.is_cuda
            ptr, ld = y_host.data_ptr(), y_host.shape[1]
        self._check(lib().esdc_sweep_host(self._h, ptr, ld, t, dt, M, K, _stream(stream)))
        return y_host

    def residual(self):
        r, yv = _D(), _D()
        rs = np.zeros(self.n_state)
        rc = lib().esdc_residual(self._h, C.byref(r), C.byref(yv), rs.ctypes.data_as(C.POINTER(_D)))
        return rc, r.value, yv.value, rs

    def stats(self, n: int) -> np.ndarray:
        out = np.zeros(n, np.int32)
        self._check(lib().esdc_stats(self._h, out.ctypes.data_as(C.POINTER(C.c_int)), n))
        return out

    def profile(self, enable: bool = True):
        self._check(lib().esdc_profile(self._h, int(enable)))

    def profile_read(self):
        """Per kernel class (setup, node, cg, residual): (milliseconds, launches)."""
        ms = (_D * 4)()
        n = (C.c_longlong * 4)()
        self._check(lib().esdc_profile_read(self._h, ms, n))
        names = ("setup", "node", "cg", "residual")
        return {names[c]: (ms[c], n[c]) for c in range(4)}

    def keep_residual(self, keep: bool = True):
        self._check(lib().esdc_keep_residual(self._h, int(keep)))

    def collocation(self, M: int, with_residual: bool = False, stream=None):
        import torch
        y = torch.empty((M, self.n_state, self.ld), dtype=torch.float64, device="cuda")
        r = torch.empty_like(y) if with_residual else None
        self._check(lib().esdc_collocation(self._h, _ptr(y), _ptr(r) if r is not None else None,
                                           _stream(stream)))
        return y, r

    def coefficients(self, z, M: int, stream=None):
        import torch
        n = z.numel()
        a = torch.empty((M, M, n), dtype=torch.float64, device="cuda")
        self._check(lib().esdc_coefficients(self._h, _ptr(z), n, M, _ptr(a), _stream(stream)))
        return a

    def debug_barrier(self, skip_block: int, limit_us: int = 0):
        """esdc_debug_barrier: make the iterative solves' grid-barrier waits run
        out (skip_block >= 0, waits limited to limit_us), or restore them (-1)."""
        self._check(lib().esdc_debug_barrier(self._h, int(skip_block), int(limit_us)))

    def diffusion_solve(self, g: float, b, x, stream=None) -> int:
        it = C.c_int()
        self._check(lib().esdc_diffusion_solve(self._h, g, _ptr(b), _ptr(x), C.byref(it), _stream(stream)))
        return it.value

    def ionic(self, y, stream=None):
        import torch
        fE, lam, yinf = (torch.empty_like(y) for _ in range(3))
        self._check(lib().esdc_ionic(self._h, _ptr(y), _ptr(fE), _ptr(lam), _ptr(yinf), _stream(stream)))
        return fE, lam, yinf


class Batch:
    """A ragged batch of tissues stepped together (``esdc_batch_*``).

    The tissues share the ionic model, chi, C_m and the options; each has its
    own mesh, scalar conductivity, stimulus and start time.  The state of the
    whole batch is one device tensor [n_state, ld]; tissue b occupies columns
    offsets[b] .. offsets[b] + n_nodes[b]."""

    def __init__(self, meshes, sigmas, chi: float, Cm: float, model: int, params, M_max: int = 8,
                 tol_cg: float = 1e-14, cg_maxit: int = 200, precond: bool = True, solver: str = "auto",
                 fuse_node1: bool = True):
        self._b = None
        L = lib()
        n = len(meshes)
        arr = (esdc_mesh * n)(*[esdc_mesh(*m) for m in meshes])
        sig = np.ascontiguousarray(sigmas, np.float64)
        opt = esdc_options()
        L.esdc_default_options(C.byref(opt))
        opt.M_max, opt.tol_cg, opt.cg_maxit, opt.precond = M_max, tol_cg, cg_maxit, int(precond)
        if solver not in ("auto", "cg", "cheb"):
            raise ValueError("solver must be 'auto', 'cg' or 'cheb'")
        opt.solver = 1 if solver == "cg" else 0
        opt.fuse_node1 = int(bool(fuse_node1))
        p = np.ascontiguousarray(params, np.float64)
        out = _VP()
        rc = L.esdc_batch_create(n, arr, sig.ctypes.data_as(C.POINTER(_D)), chi, Cm, model,
                                 p.ctypes.data_as(C.POINTER(_D)), len(p), C.byref(opt), C.byref(out))
        if rc != ESDC_OK:
            raise EsdcError(rc, "esdc_batch_create failed")
        self._b = out.value
        self.n = n
        ns, ld = C.c_int(), _I64()
        offs = np.zeros(n, np.int64)
        self._check(L.esdc_batch_layout(self._b, C.byref(ns), C.byref(ld), offs.ctypes.data_as(C.POINTER(_I64))))
        self.n_state, self.ld, self.offsets = ns.value, ld.value, offs
        self.n_nodes = np.array([m[1] * m[2] * m[3] for m in meshes], np.int64)

    @classmethod
    def from_workloads(cls, wls, **kw) -> "Batch":
        """All workloads must share model, parameters, chi and C_m."""
        w0 = wls[0]
        meshes = [(w.dim, w.nx, w.ny, w.nz, w.h) for w in wls]
        b = cls(meshes, [w.sigma for w in wls], w0.chi, w0.Cm, w0.model, w0.params, **kw)
        for k, w in enumerate(wls):
            b.set_stimulus(k, w.boxes, w.amp, w.t_on, w.t_off)
        return b

    def _check(self, rc: int):
        if rc != ESDC_OK:
            msg = lib().esdc_batch_last_error(self._b).decode() if self._b else ""
            raise EsdcError(rc, msg)

    def close(self):
        if self._b:
            lib().esdc_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stimulus(self, tissue: int, boxes, amp, t_on, t_off):
        box = np.ascontiguousarray(np.asarray(boxes, np.int32).reshape(-1))
        a, on, off = (np.ascontiguousarray(v, np.float64) for v in (amp, t_on, t_off))
        self._check(lib().esdc_batch_set_stimulus(self._b, tissue, len(a), box.ctypes.data_as(C.POINTER(C.c_int)),
                                                  a.ctypes.data_as(C.POINTER(_D)), on.ctypes.data_as(C.POINTER(_D)),
                                                  off.ctypes.data_as(C.POINTER(_D))))

    def new_state(self):
        import torch
        return torch.zeros((self.n_state, self.ld), dtype=torch.float64, device="cuda")

    def init_state(self, y, V0: float, stream=None):
        self._check(lib().esdc_batch_init_state(self._b, _ptr(y), V0, _stream(stream)))

    def sweep(self, y, t, dt: float, M: int, K: int, stream=None):
        tv = np.ascontiguousarray(np.broadcast_to(np.asarray(t, np.float64), (self.n,)))
        self._check(lib().esdc_batch_sweep(self._b, _ptr(y), tv.ctypes.data_as(C.POINTER(_D)), dt, M, K,
                                           _stream(stream)))

    def sweep_from(self, y_in, y_out, t, dt: float, M: int, K: int, from_iterate: bool, stream=None):
        tv = np.ascontiguousarray(np.broadcast_to(np.asarray(t, np.float64), (self.n,)))
        self._check(lib().esdc_batch_sweep_from(self._b, _ptr(y_in), _ptr(y_out), tv.ctypes.data_as(C.POINTER(_D)),
                                                dt, M, K, int(from_iterate), _stream(stream)))

    def qpar(self, y_in, y_out, t0: float, dt: float, M: int, iters: int, stream=None):
        """Q^par iterations over the batch's tissues as time slices (esdc_batch_qpar)."""
        self._check(lib().esdc_batch_qpar(self._b, _ptr(y_in), _ptr(y_out), t0, dt, M, iters, _stream(stream)))

    def iterate(self, M: int):
        """The batch's collocation iterate y_{n,1..M} as a tensor view [M, n_state, ld] (device memory
        owned by the batch)."""
        import torch
        Y = _VP()
        self._check(lib().esdc_batch_iterate(self._b, C.byref(Y), None))
        return _device_view(Y.value, (M, self.n_state, self.ld))

    def residual(self):
        """(return code, res_inf[n], y_inf[n]); does not raise on solver flags."""
        r = np.zeros(self.n)
        y = np.zeros(self.n)
        rc = lib().esdc_batch_residual(self._b, r.ctypes.data_as(C.POINTER(_D)), y.ctypes.data_as(C.POINTER(_D)))
        return rc, r, y

    def stats(self, K: int, M: int) -> np.ndarray:
        out = np.zeros(K * M * self.n, np.int32)
        self._check(lib().esdc_batch_stats(self._b, out.ctypes.data_as(C.POINTER(C.c_int)), len(out)))
        return out.reshape(K * M, self.n)

    def set_graph(self, on: bool):
        self._check(lib().esdc_batch_set_graph(self._b, int(on)))

    def graph_active(self) -> bool:
        return bool(lib().esdc_batch_graph_active(self._b))

    def graph_error(self) -> str:
        return lib().esdc_batch_graph_error(self._b).decode()

    def set_shape(self, node_waves: int, cg_threads: int, cg_blocks_per_sm: int):
        self._check(lib().esdc_batch_set_shape(self._b, node_waves, cg_threads, cg_blocks_per_sm))

    def shape(self):
        w, t, b = C.c_int(), C.c_int(), C.c_int()
        self._check(lib().esdc_batch_get_shape(self._b, C.byref(w), C.byref(t), C.byref(b)))
        return w.value, t.value, b.value

    def set_persistent(self, on: bool, threads: int = 512, tile: int = 128):
        """esdc_batch_set_persistent: one persistent launch per step (on) or the launch sequence."""
        self._check(lib().esdc_batch_set_persistent(self._b, int(on), int(threads), int(tile)))

    def persistent(self):
        """(on, threads, tile) of the persistent launch."""
        o, t, n = C.c_int(), C.c_int(), C.c_int()
        self._check(lib().esdc_batch_get_persistent(self._b, C.byref(o), C.byref(t), C.byref(n)))
        return bool(o.value), t.value, n.value

    def tune(self, y_scratch, V0: float, t: float, dt: float, M: int, K: int, reps: int = 3, stream=None):
        self._check(lib().esdc_batch_tune(self._b, _ptr(y_scratch), V0, t, dt, M, K, reps, _stream(stream)))

    def tissue(self, y, b: int):
        """View of tissue b's columns of a batch state."""
        o = int(self.offsets[b])
        return y[:, o:o + int(self.n_nodes[b])]


def _device_view(ptr: int, shape):
    """A float64 CUDA tensor viewing library-owned device memory (no copy)."""
    import torch

    class _Arr:
        pass
    a = _Arr()
    n = int(np.prod(shape))
    a.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (int(ptr), False), "version": 2,
                                  "strides": None}
    return torch.as_tensor(a, device="cuda").view(*shape)


def hsdc2(fine: "Batch", coarse, y_in, y_out, t0: float, dt: float, M1: int, M2: int, iters: int, stream=None):
    """Two-level Algorithm HSDC over the fine batch's tissues as time slices
    (esdc_hsdc2); coarse is a list of single-tissue batches, one per slice."""
    arr = (_VP * len(coarse))(*[c._b for c in coarse])
    rc = lib().esdc_hsdc2(fine._b, arr, _ptr(y_in), _ptr(y_out), t0, dt, M1, M2, iters, _stream(stream))
    fine._check(rc)


def hsdc(levels, coarse, y_in, y_out, t0: float, dt: float, Ms, iters: int, stream=None):
    """Algorithm HSDC with L = len(Ms) levels (esdc_hsdc): levels is a list of
    L - 1 batches of the same P slices (the Q^par levels, finest first), coarse
    a list of P single-tissue batches (the Q^seq level)."""
    lv = (_VP * len(levels))(*[b._b for b in levels])
    arr = (_VP * len(coarse))(*[c._b for c in coarse])
    m = (C.c_int * len(Ms))(*[int(x) for x in Ms])
    rc = lib().esdc_hsdc(lv, arr, m, len(Ms), _ptr(y_in), _ptr(y_out), t0, dt, iters, _stream(stream))
    levels[0]._check(rc)


def sensor_traces(solver: "Solver", sigma, g_na, g_k, y0, t0: float, dt: float, M: int, K: int, nsteps: int, sens):
    """V at the sensor nodes after each of nsteps HSDC steps from y0, as a
    differentiable function of the conductivity field sigma [N] and the maximal
    conductances g_Na, g_K (0-d tensors): the backward pass is the library's
    discrete adjoint (esdc_adjoint_backward), with one checkpoint per step."""
    import torch

    class _Traces(torch.autograd.Function):
        @staticmethod
        def forward(ctx, sig, gna, gk):
            p = solver.params.copy()
            p[0], p[1] = float(gna), float(gk)
            solver.set_params(p)
            solver.set_conductivity_field(sig.detach().cpu().numpy())
            y = y0.clone()
            traces = torch.empty((nsteps, sens.numel()), dtype=torch.float64, device="cuda")
            ckpt = torch.empty((nsteps, solver.n_state, solver.ld), dtype=torch.float64, device="cuda")
            solver.adjoint_forward(y, t0, dt, M, K, nsteps, sens, traces, ckpt)
            ctx.ckpt = ckpt
            ctx.sig_device = sig.device
            return traces

        @staticmethod
        def backward(ctx, dtr):
            gsig, gpar, _ = solver.adjoint_backward(ctx.ckpt, t0, dt, M, K, nsteps, sens, dtr.contiguous())
            one = torch.ones((), dtype=torch.float64)
            return gsig.to(ctx.sig_device), one * gpar[0], one * gpar[1]

    return _Traces.apply(sigma, g_na, g_k)
