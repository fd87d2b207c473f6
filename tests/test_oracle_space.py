"""Pins of the oracle's Laplacian and linear solves (Sec. 2.2 space
discretisation; Sec. 5 DCT-II solver) against closed-form cosine modes and
dense linear algebra."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_19994_gb300 import inputs as I


def _mono(nx, ny, nz, h=0.3, solver=O.SOLVE_DCT):
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.h = h
    return O.Monodomain(wl, solver=solver)


def _mode(nx, ny, nz, kx, ky, kz):
    ix = np.arange(nx)[None, None, :]
    iy = np.arange(ny)[None, :, None]
    iz = np.arange(nz)[:, None, None]
    v = (np.cos(np.pi * kx * (ix + 0.5) / nx) * np.cos(np.pi * ky * (iy + 0.5) / ny)
         * np.cos(np.pi * kz * (iz + 0.5) / nz))
    return v.reshape(-1)


@pytest.mark.parametrize("shape,k", [((7, 1, 1), (3, 0, 0)), ((6, 5, 1), (2, 4, 0)),
                                     ((5, 4, 3), (1, 3, 2)), ((9, 8, 4), (0, 0, 0))])
def test_laplacian_cosine_eigenmodes(orc, shape, k):
    # cos(pi k (i+1/2)/n) is an eigenvector of the mirrored-ghost stencil with
    # eigenvalue -(4/h^2) sin^2(pi k / (2n)) per axis.
    nx, ny, nz = shape
    m = _mono(nx, ny, nz, h=0.3)
    v = _mode(nx, ny, nz, *k)
    mu = sum(-(4 / 0.09) * np.sin(np.pi * kk / (2 * n)) ** 2 for kk, n in zip(k, shape))
    np.testing.assert_allclose(m.laplacian(v), mu * v, atol=1e-12 * max(1, abs(mu)))


def test_laplacian_dense_properties(orc):
    # symmetric, negative semi-definite, null space = constants
    nx, ny, nz = 5, 4, 3
    m = _mono(nx, ny, nz, h=0.5)
    N = nx * ny * nz
    L = np.stack([m.laplacian(e) for e in np.eye(N)], axis=1)
    np.testing.assert_allclose(L, L.T, atol=1e-14)
    ev = np.linalg.eigvalsh(L)
    assert ev.max() < 1e-12 and abs(ev[-1]) < 1e-12 and ev[-2] < -1e-3
    np.testing.assert_allclose(L @ np.ones(N), 0.0, atol=1e-13)
    assert abs(np.diag(L)).max() <= 6 / 0.25 + 1e-12


@pytest.mark.parametrize("shape", [(12, 1, 1), (9, 7, 1), (6, 5, 4)])
def test_solvers_agree_and_solve(orc, shape):
    nx, ny, nz = shape
    m = _mono(nx, ny, nz, h=0.25)
    rng = np.random.default_rng(1)
    b = rng.normal(size=nx * ny * nz)
    g = 0.0123
    xs = [m.solve_shifted(g, b, method=meth) for meth in (O.SOLVE_DCT, O.SOLVE_CG, O.SOLVE_DENSE)]
    for x in xs:
        r = x - g * m.laplacian(x) - b
        assert np.abs(r).max() < 1e-13 * np.abs(b).max()
    np.testing.assert_allclose(xs[0], xs[2], atol=1e-13)
    np.testing.assert_allclose(xs[1], xs[2], atol=1e-13)
