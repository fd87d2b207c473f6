"""The C-ABI library loads without a GPU, exports every entry point that
include/esdc.h declares, and rejects invalid arguments before touching CUDA."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2405_19994_gb300 import build as B
    B.build()
    from paper_2405_19994_gb300 import esdc
    return esdc.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "esdc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(esdc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("esdc_create", "esdc_sweep", "esdc_residual", "esdc_destroy", "esdc_set_stimulus",
                 "esdc_state_size", "esdc_init_state", "esdc_stats", "esdc_last_error", "esdc_sweep_host"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_invalid_arguments_rejected_without_gpu(L):
    from paper_2405_19994_gb300 import esdc as E
    from paper_2405_19994_gb300 import inputs as I
    p = I.hh1952_params()
    pp = p.ctypes.data_as(C.POINTER(C.c_double))
    out = C.c_void_p(1)

    def create(mesh, sigma=0.17, chi=140.0, Cm=0.01, model=0, params=pp, n=7, optp=None):
        return L.esdc_create(C.byref(mesh), sigma, chi, Cm, model, params, n, optp, C.byref(out))

    ok = E.esdc_mesh(2, 8, 8, 1, 0.25)
    assert create(E.esdc_mesh(0, 8, 8, 1, 0.25)) == -1 and out.value is None
    assert create(E.esdc_mesh(2, 0, 8, 1, 0.25)) == -1
    assert create(E.esdc_mesh(2, 8, 8, 3, 0.25)) == -1          # 2D with nz != 1
    assert create(E.esdc_mesh(1, 8, 2, 1, 0.25)) == -1          # 1D with ny != 1
    assert create(E.esdc_mesh(2, 8, 8, 1, 0.0)) == -1
    assert create(E.esdc_mesh(2, 8, 8, 1, float("nan"))) == -1
    assert create(E.esdc_mesh(3, 70000, 70000, 1, 0.1)) == -1   # more than 2^31 nodes
    assert create(ok, chi=0.0) == -1
    assert create(ok, Cm=-1.0) == -1
    assert create(ok, model=7) == -1
    assert create(ok, n=6) == -1                                # HH needs 7 parameters
    assert create(ok, params=None) == -1
    bad = p.copy(); bad[2] = np.inf
    assert create(ok, params=bad.ctypes.data_as(C.POINTER(C.c_double))) == -1
    opt = E.esdc_options(); L.esdc_default_options(C.byref(opt))
    assert (opt.M_max, opt.tol_cg, opt.cg_maxit, opt.precond, opt.precision, opt.solver, opt.fuse_node1) == \
        (8, 1e-14, 200, 1, 0, 0, 1)
    opt.precision = 2
    assert create(ok, optp=C.byref(opt)) == -1
    opt.precision = 0
    opt.solver = 4
    assert create(ok, optp=C.byref(opt)) == -1
    opt.solver = 2; opt.precision = 1                           # the DCT solve is FP64
    assert create(ok, optp=C.byref(opt)) == -6
    opt.solver = 0; opt.precision = 0
    opt.M_max = 9
    assert create(ok, optp=C.byref(opt)) == -1
    opt.M_max = 4; opt.cg_maxit = 0
    assert create(ok, optp=C.byref(opt)) == -1
    opt.cg_maxit = 200; opt.fuse_node1 = 2
    assert create(ok, optp=C.byref(opt)) == -1
    # null handles
    assert L.esdc_sweep(None, None, 0.0, 0.1, 3, 4, None) == -1
    assert L.esdc_residual(None, None, None, None) == -1
    assert L.esdc_state_size(None, None, None, None) == -1
    L.esdc_destroy(None)
    assert L.esdc_last_error(None) == b"null handle"


def test_no_product_import_of_the_oracle():
    # The product path (package + C sources) must never reach the oracle.
    pkg = os.path.join(ROOT, "paper_2405_19994_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "esdc_oracle" not in txt and "liborc" not in txt, f


def test_batch_invalid_arguments_rejected_without_gpu(L):
    from paper_2405_19994_gb300 import esdc as E
    from paper_2405_19994_gb300 import inputs as I
    p = I.hh1952_params()
    pp = p.ctypes.data_as(C.POINTER(C.c_double))
    out = C.c_void_p(1)
    meshes = (E.esdc_mesh * 2)(E.esdc_mesh(2, 8, 8, 1, 0.25), E.esdc_mesh(2, 5, 3, 1, 0.25))
    sig = np.array([0.1, 0.2])
    sp = sig.ctypes.data_as(C.POINTER(C.c_double))

    def create(n=2, m=meshes, s=sp, chi=140.0, Cm=0.01, model=0, params=pp, npar=7, optp=None):
        return L.esdc_batch_create(n, m, s, chi, Cm, model, params, npar, optp, C.byref(out))

    assert create(n=0) == -1 and out.value is None
    assert create(m=None) == -1
    assert create(s=None) == -1
    assert create(chi=0.0) == -1
    assert create(npar=6) == -1
    bad = np.array([0.1, -1.0])
    assert create(s=bad.ctypes.data_as(C.POINTER(C.c_double))) == -1
    bm = (E.esdc_mesh * 2)(E.esdc_mesh(2, 8, 8, 3, 0.25), E.esdc_mesh(2, 5, 3, 1, 0.25))
    assert create(m=bm) == -1                                  # 2D mesh with nz != 1
    opt = E.esdc_options(); L.esdc_default_options(C.byref(opt))
    opt.precision = 1
    assert create(optp=C.byref(opt)) == -6                     # batches run the FP64 path
    opt.precision = 0
    for bad_solver in (2, 4):                                  # batches: automatic (0, 3) or CG
        opt.solver = bad_solver
        assert create(optp=C.byref(opt)) == -1
    assert L.esdc_batch_sweep(None, None, None, 0.1, 3, 4, None) == -1
    assert L.esdc_batch_residual(None, None, None) == -1
    assert L.esdc_batch_layout(None, None, None, None) == -1
    L.esdc_batch_destroy(None)
    assert L.esdc_batch_last_error(None) == b"null batch"


def test_later_entry_points_reject_invalid_arguments_without_gpu(L):
    D = C.POINTER(C.c_double)
    # null handles
    assert L.esdc_set_stencil_order(None, 4) == -1
    assert L.esdc_get_solver(None, None) == -1
    assert L.esdc_set_conductivity_field(None, None) == -1
    assert L.esdc_set_conductivity_layers(None, None, None, None, None) == -1
    assert L.esdc_set_params(None, None, 7) == -1
    assert L.esdc_adjoint_forward(None, None, 0.0, 0.1, 3, 4, 1, 0, None, None, None, None) == -1
    assert L.esdc_adjoint_backward(None, None, 0.0, 0.1, 3, 4, 1, 0, None, None, None, None, None, None,
                                   None) == -1
    assert L.esdc_batch_sweep_ex(None, None, None, None, None, 0.1, 3, 1, 0, 0, None) == -1
    assert L.esdc_batch_sweep_from(None, None, None, None, 0.1, 3, 1, 0, None) == -1
    assert L.esdc_batch_qpar(None, None, None, 0.0, 0.1, 3, 2, None) == -1
    assert L.esdc_batch_iterate(None, None, None) == -1
    assert L.esdc_debug_barrier(None, 0, 1000) == -1
    assert L.esdc_hsdc2(None, None, None, None, 0.0, 0.1, 3, 2, 1, None) == -1
    nolev = (C.c_void_p * 1)(None)
    ms = (C.c_int * 2)(3, 2)
    assert L.esdc_hsdc(None, None, ms, 2, None, None, 0.0, 0.1, 1, None) == -1
    assert L.esdc_hsdc(nolev, None, ms, 2, None, None, 0.0, 0.1, 1, None) == -1
    d1, d2 = C.c_double(), C.c_double()
    assert L.esdc_fma_probe(2, 10, C.byref(d1), C.byref(d2), None) == -1
    assert L.esdc_fma_probe(0, 0, C.byref(d1), C.byref(d2), None) == -1
    assert L.esdc_fma_probe(0, 10, None, C.byref(d2), None) == -1
    assert L.esdc_batch_set_shape(None, 1, 512, 1) == -1
    assert L.esdc_batch_tune(None, None, -75.0, 0.0, 0.1, 3, 4, 1, None) == -1
    assert L.esdc_batch_graph_active(None) == 0
    # the node interpolator: null arrays, too many rows, equal source and destination
    W = np.eye(2)
    Wp = W.ctypes.data_as(D)
    src, dst = C.c_void_p(16), C.c_void_p(32)
    assert L.esdc_interp(None, 2, 4, dst, 2, 4, 1, 4, Wp, 0.0, None) == -1
    assert L.esdc_interp(src, 9, 4, dst, 2, 4, 1, 4, Wp, 0.0, None) == -1
    assert L.esdc_interp(src, 2, 4, src, 2, 4, 1, 4, Wp, 0.0, None) == -1
    assert L.esdc_interp(src, 2, 2, dst, 2, 4, 1, 4, Wp, 0.0, None) == -1     # pitch shorter than the columns
    bad = np.array([[1.0, np.nan], [0.0, 1.0]])
    assert L.esdc_interp(src, 2, 4, dst, 2, 4, 1, 4, bad.ctypes.data_as(D), 0.0, None) == -1
    assert L.esdc_interp(src, 2, 4, dst, 2, 4, 1, 0, Wp, 0.0, None) == 0      # nothing to do


def test_exp_table_entries_are_correctly_rounded():
    # esdc_exp's table: 2^(j/2048) for j = 0..2047, each within half an ulp of
    # the exact value (here computed as a decimal power at 40 digits)
    import decimal
    import re
    src = open(os.path.join(ROOT, "paper_2405_19994_gb300", "csrc", "esdc_exp_table.h")).read()
    vals = [float.fromhex(v) for v in re.findall(r"0x[0-9a-f.]+p[+-]\d+", src[src.index("{"):])]
    assert len(vals) == 2048
    decimal.getcontext().prec = 40
    for j, v in enumerate(vals):
        exact = decimal.Decimal(2) ** (decimal.Decimal(j) / 2048)
        ulp = math.ulp(v)
        assert abs(decimal.Decimal(v) - exact) <= decimal.Decimal(ulp) / 2, j
