"""The build-time accuracy of the tables the kernels evaluate instead of
transcendental functions, checked on the host (esdc_table_errors: no device
work).  The gate table in V (w_inf and Lambda of every gate, as Lambda and
b = -Lambda w_inf) and the set-up's coefficient table in z = dt Lambda (dt S_ij,
dt d_i phi_1) must reproduce their long-double evaluations to within a few
units of 1e-16; a handle refuses a table above 4e-15 and evaluates directly."""
import ctypes as C

import numpy as np
import pytest

from paper_2405_19994_gb300 import esdc as E
from paper_2405_19994_gb300 import inputs as I


@pytest.fixture(scope="module")
def L():
    return E.lib()


def errors(L, model, params, M, dt):
    p = np.ascontiguousarray(params, np.float64)
    err = (C.c_double * 3)()
    rc = L.esdc_table_errors(model, p.ctypes.data_as(C.POINTER(C.c_double)), len(p), M, dt, err)
    return rc, list(err)


@pytest.mark.parametrize("model,params", [(I.MODEL_SYN19, I.syn19_params()), (I.MODEL_HH1952, I.hh1952_params()),
                                          (I.MODEL_HH1952, I.hh1952_params(v_rest=-65.0))])
def test_gate_table_at_rounding_level(L, model, params):
    rc, err = errors(L, model, params, 4, 0.05)
    assert rc == 0
    assert err[0] < 1e-15 and err[1] < 1e-15, err


@pytest.mark.parametrize("M", range(1, 9))
@pytest.mark.parametrize("dt", [1e-3, 0.05, 1.0])
def test_setup_coefficient_table_within_tolerance(L, M, dt):
    rc, err = errors(L, I.MODEL_HH1952, I.hh1952_params(), M, dt)
    assert rc == 0
    # measured: 6.6e-16 for M = 4, 1.4e-15 and 1.5e-15 for M = 1, 2, 2.0e-15 for
    # M = 8 (larger B coefficients), independent of dt
    assert err[2] < 2.5e-15, (M, dt, err[2])


def test_table_errors_rejects_bad_arguments(L):
    p = np.ascontiguousarray(I.hh1952_params(), np.float64)
    ptr = p.ctypes.data_as(C.POINTER(C.c_double))
    err = (C.c_double * 3)()
    assert L.esdc_table_errors(I.MODEL_HH1952, ptr, len(p), 0, 0.05, err) == -1        # M
    assert L.esdc_table_errors(I.MODEL_HH1952, ptr, len(p), 9, 0.05, err) == -1
    assert L.esdc_table_errors(I.MODEL_HH1952, ptr, len(p), 3, 0.0, err) == -1         # dt
    assert L.esdc_table_errors(I.MODEL_HH1952, ptr, len(p) - 1, 3, 0.05, err) == -1    # parameter count
    assert L.esdc_table_errors(7, ptr, len(p), 3, 0.05, err) == -1                    # model
    assert L.esdc_table_errors(I.MODEL_HH1952, ptr, len(p), 3, 0.05, None) == -1
