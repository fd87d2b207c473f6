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


@pytest.mark.parametrize("shape", [(8, 1, 1), (4, 6, 1), (8, 3, 5), (1, 1, 1)])
def test_shifted_operator_spectrum_interval(orc, shape):
    # The whole spectrum of I - g L lies in [1, 1 + (g/h^2) sum_axes 4 sin^2(pi (n-1)/(2n))]
    # and reaches both ends: the interval a Chebyshev semi-iteration on this
    # operator is built on.  Dense eigenvalues of the oracle's operator.
    nx, ny, nz = shape
    h, g = 0.3, 0.07
    m = _mono(nx, ny, nz, h=h)
    N = nx * ny * nz
    B = np.stack([e - g * m.laplacian(e) for e in np.eye(N)], axis=1)
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    hi = 1 + g / h**2 * sum(4 * np.sin(np.pi * (n - 1) / (2 * n)) ** 2 for n in shape)
    assert abs(ev.min() - 1.0) < 1e-12 and abs(ev.max() - hi) < 1e-12 * hi


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


# ---------------------------------------------------------------- layered anisotropic conductivity

def _aniso(nx, ny, nz, h=0.3, sl=0.17, st=0.02):
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.h = h
    wl.layers = I.fibre_layers(nz, sl, st)
    return wl, O.Monodomain(wl, solver=O.SOLVE_CG)


def test_aniso_operator_exact_on_quadratics(orc):
    # Interior nodes: central differences are exact for quadratics, so
    # A x^2 = 2 sxx, A y^2 = 2 syy, A (x y) = 2 sxy, A z^2 = 2 szz (per layer).
    nx, ny, nz, h = 9, 8, 7, 0.3
    wl, m = _aniso(nx, ny, nz, h)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = ((ix + 0.5) * h).transpose(2, 1, 0).reshape(-1)
    y = ((iy + 0.5) * h).transpose(2, 1, 0).reshape(-1)
    z = ((iz + 0.5) * h).transpose(2, 1, 0).reshape(-1)
    kz = iz.transpose(2, 1, 0).reshape(-1)
    inner = ((ix > 0) & (ix < nx - 1) & (iy > 0) & (iy < ny - 1) & (iz > 0) & (iz < nz - 1)).transpose(2, 1, 0).reshape(-1)
    L = wl.layers
    for f, want in ((x * x, 2 * L["sxx"][kz]), (y * y, 2 * L["syy"][kz]), (x * y, 2 * L["sxy"][kz]),
                    (z * z, 2 * L["szz"][kz])):
        got = m.conductivity(f)
        np.testing.assert_allclose(got[inner], want[inner], rtol=0, atol=1e-11)


def test_aniso_operator_symmetric_nsd_constant_nullspace(orc):
    nx, ny, nz = 6, 5, 4
    wl, m = _aniso(nx, ny, nz, h=0.5, sl=0.3, st=0.01)       # strong anisotropy
    N = nx * ny * nz
    A = np.stack([m.conductivity(e) for e in np.eye(N)], axis=1)
    np.testing.assert_allclose(A, A.T, atol=1e-14)
    ev = np.linalg.eigvalsh(A)
    assert ev.max() < 1e-12 and ev[-2] < -1e-4
    np.testing.assert_allclose(A @ np.ones(N), 0.0, atol=1e-13)


@pytest.mark.parametrize("sl,st", [(0.17, 0.02), (0.3, 0.01)])
def test_aniso_spectrum_inside_gershgorin_interval(orc, sl, st):
    # The interval a Chebyshev semi-iteration on I - g A is built on for the
    # layered operator: the smallest eigenvalue of I - g A is 1 (constants), the
    # largest at most 1 + g G with G = max over layers of
    # (4 sxx + 4 syy + 2|sxy| + 2 (faces' szz means))/h^2 (Gershgorin).
    nx, ny, nz, h, g = 6, 5, 4, 0.4, 0.3
    wl, m = _aniso(nx, ny, nz, h, sl=sl, st=st)
    N = nx * ny * nz
    B = np.stack([e - g * m.conductivity(e) for e in np.eye(N)], axis=1)
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    L = wl.layers
    face = np.append(0.5 * (L["szz"][:-1] + L["szz"][1:]), 0.0)            # face k | k+1
    below = np.insert(face[:-1], 0, 0.0)
    G = np.max(4 * L["sxx"] + 4 * L["syy"] + 2 * np.abs(L["sxy"]) + 2 * (face + below)) / h**2
    assert abs(ev.min() - 1.0) < 1e-12
    assert ev.max() <= 1 + g * G + 1e-12
    assert ev.max() >= 1 + 0.6 * g * G                                      # and the bound is not loose


def test_aniso_reduces_to_isotropic(orc):
    nx, ny, nz = 7, 6, 3
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    iso = O.Monodomain(wl)
    wl2 = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl2.layers = {"sxx": np.full(nz, wl.sigma), "syy": np.full(nz, wl.sigma), "sxy": np.zeros(nz),
                  "szz": np.full(nz, wl.sigma)}
    lay = O.Monodomain(wl2, solver=O.SOLVE_CG)
    v = np.random.default_rng(3).normal(size=nx * ny * nz)
    np.testing.assert_allclose(lay.conductivity(v), wl.sigma * iso.laplacian(v), rtol=0, atol=1e-12)


def test_aniso_solves_agree(orc):
    wl, m = _aniso(8, 7, 5)
    b = np.random.default_rng(4).normal(size=8 * 7 * 5)
    g = 0.02
    x_cg = m.solve_A(g, b, method=O.SOLVE_CG)
    x_de = m.solve_A(g, b, method=O.SOLVE_DENSE)
    np.testing.assert_allclose(x_cg, x_de, atol=1e-13)
    r = x_cg - g * m.conductivity(x_cg) - b
    assert np.abs(r).max() < 1e-13


def test_aniso_second_order_consistency(orc):
    # smooth field, interior nodes: error of A f against div(sigma grad f) falls ~4x per halving of h
    errs = []
    for n, h in ((12, 0.2), (24, 0.1)):
        wl, m = _aniso(n, n, 3, h)
        ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(3), indexing="ij")
        x = ((ix + 0.5) * h).transpose(2, 1, 0).reshape(-1)
        y = ((iy + 0.5) * h).transpose(2, 1, 0).reshape(-1)
        kz = iz.transpose(2, 1, 0).reshape(-1)
        f = np.sin(1.3 * x) * np.cos(0.7 * y)
        fxx = -1.69 * f
        fyy = -0.49 * f
        fxy = -1.3 * 0.7 * np.cos(1.3 * x) * np.sin(0.7 * y)
        L = wl.layers
        want = L["sxx"][kz] * fxx + L["syy"][kz] * fyy + 2 * L["sxy"][kz] * fxy
        inner = ((ix > 0) & (ix < n - 1) & (iy > 0) & (iy < n - 1) & (iz == 1)).transpose(2, 1, 0).reshape(-1)
        errs.append(np.abs(m.conductivity(f) - want)[inner].max())
    assert 3.3 < errs[0] / errs[1] < 4.8, errs


# ---------------------------------------------------------------- per-node conductivity field

def _field(nx, ny, nz, h=0.3, field=None, seed=0):
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.h = h
    wl.sigma_field = (I.lognormal_field(nx, ny, nz, seed=seed, corr=2.0) if field is None
                      else np.asarray(field, np.float64))
    return wl, O.Monodomain(wl, solver=O.SOLVE_CG)


def test_field_constant_is_scalar_sigma(orc):
    nx, ny, nz = 7, 6, 3
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    iso = O.Monodomain(wl)
    _, fm = _field(nx, ny, nz, h=wl.h, field=np.full(nx * ny * nz, 0.23))
    v = np.random.default_rng(5).normal(size=nx * ny * nz)
    np.testing.assert_allclose(fm.conductivity(v), 0.23 * iso.laplacian(v), rtol=0, atol=1e-12)


def test_field_operator_symmetric_nsd_constant_nullspace(orc):
    nx, ny, nz = 6, 5, 3
    wl, m = _field(nx, ny, nz, h=0.5, seed=2)
    N = nx * ny * nz
    A = np.stack([m.conductivity(e) for e in np.eye(N)], axis=1)
    np.testing.assert_allclose(A, A.T, atol=1e-14)
    ev = np.linalg.eigvalsh(A)
    assert ev.max() < 1e-12 and ev[-2] < -1e-4
    np.testing.assert_allclose(A @ np.ones(N), 0.0, atol=1e-13)
    # brute force: sum over the faces of the quadratic form, face sigma = mean of its two nodes
    v = np.random.default_rng(6).normal(size=N)
    s = wl.sigma_field
    q = 0.0
    for p in range(N):
        ix, iy, iz = p % nx, (p // nx) % ny, p // (nx * ny)
        for d, ok in ((1, ix < nx - 1), (nx, iy < ny - 1), (nx * ny, iz < nz - 1)):
            if ok:
                q -= 0.5 * (s[p] + s[p + d]) * (v[p + d] - v[p]) ** 2
    assert abs(v @ A @ v - q / 0.25) < 1e-10 * abs(q)


def test_field_second_order_consistency(orc):
    # div(sigma grad f) for smooth sigma and f, interior nodes: error falls ~4x per halving of h
    errs = []
    for n, h in ((16, 0.2), (32, 0.1)):
        ix, iy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        x = (ix + 0.5) * h
        y = (iy + 0.5) * h
        sig = 0.1 + 0.05 * np.sin(0.9 * x) * np.cos(0.6 * y)
        f = np.cos(1.1 * x) * np.sin(0.8 * y)
        wl, m = _field(n, n, 1, h=h, field=sig.reshape(-1))
        sx = 0.05 * 0.9 * np.cos(0.9 * x) * np.cos(0.6 * y)
        sy = -0.05 * 0.6 * np.sin(0.9 * x) * np.sin(0.6 * y)
        fx = -1.1 * np.sin(1.1 * x) * np.sin(0.8 * y)
        fy = 0.8 * np.cos(1.1 * x) * np.cos(0.8 * y)
        lapf = -(1.21 + 0.64) * f
        want = sig * lapf + sx * fx + sy * fy
        got = m.conductivity(f.reshape(-1)).reshape(n, n)
        errs.append(np.abs(got - want)[1:-1, 1:-1].max())
    assert 3.3 < errs[0] / errs[1] < 4.8, errs


def test_field_solves_agree(orc):
    wl, m = _field(8, 7, 2, seed=3)
    b = np.random.default_rng(4).normal(size=8 * 7 * 2)
    g = 0.03
    x_cg = m.solve_A(g, b, method=O.SOLVE_CG)
    x_de = m.solve_A(g, b, method=O.SOLVE_DENSE)
    np.testing.assert_allclose(x_cg, x_de, atol=1e-13)
    assert np.abs(x_cg - g * m.conductivity(x_cg) - b).max() < 1e-13


# ---------------------------------------------------------------- fourth-order Laplacian (the paper's scheme)

def _mono4(nx, ny, nz, h=0.3, solver=O.SOLVE_DCT):
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.h = h
    wl.order = 4
    return O.Monodomain(wl, solver=solver)


@pytest.mark.parametrize("shape,k", [((7, 1, 1), (3, 0, 0)), ((6, 5, 1), (2, 4, 0)), ((5, 4, 3), (1, 3, 2)),
                                     ((2, 3, 1), (1, 2, 0)), ((9, 8, 4), (0, 0, 0))])
def test_laplacian4_cosine_eigenmodes(orc, shape, k):
    # cos(pi k (i+1/2)/n) is an eigenvector of the mirrored five-point stencil
    # with eigenvalue (32 cos t - 2 cos 2t - 30)/(12 h^2), t = pi k/n, per axis
    nx, ny, nz = shape
    m = _mono4(nx, ny, nz, h=0.3)
    v = _mode(nx, ny, nz, *k)
    mu = sum((32 * np.cos(np.pi * kk / n) - 2 * np.cos(2 * np.pi * kk / n) - 30) / (12 * 0.09) if n > 1 else 0.0
             for kk, n in zip(k, shape))
    np.testing.assert_allclose(m.laplacian(v), mu * v, atol=1e-12 * max(1, abs(mu)))


def test_laplacian4_symmetric_nsd_constant_nullspace(orc):
    nx, ny, nz = 6, 4, 3
    m = _mono4(nx, ny, nz, h=0.5)
    N = nx * ny * nz
    L = np.stack([m.laplacian(e) for e in np.eye(N)], axis=1)
    np.testing.assert_allclose(L, L.T, atol=1e-13)
    ev = np.linalg.eigvalsh(L)
    assert ev.max() < 1e-12 and ev[-2] < -1e-3
    np.testing.assert_allclose(L @ np.ones(N), 0.0, atol=1e-13)


def test_laplacian4_fourth_order_consistency(orc):
    # interior nodes (two cells from the boundary): the error against the exact
    # Laplacian falls ~16x per halving of h (it is ~4x for the 5-point stencil)
    errs = []
    for n, h in ((16, 0.2), (32, 0.1)):
        ix, iy = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        x, y = (ix + 0.5) * h, (iy + 0.5) * h
        f = np.sin(1.3 * x) * np.cos(0.7 * y)
        m = _mono4(n, n, 1, h=h)
        got = m.laplacian(f.reshape(-1)).reshape(n, n)
        errs.append(np.abs(got - (-(1.69 + 0.49) * f))[2:-2, 2:-2].max())
    assert 13.0 < errs[0] / errs[1] < 19.0, errs


@pytest.mark.parametrize("shape", [(12, 1, 1), (9, 7, 1), (6, 5, 4), (2, 3, 2)])
def test_laplacian4_solvers_agree_and_solve(orc, shape):
    nx, ny, nz = shape
    m = _mono4(nx, ny, nz, h=0.25)
    b = np.random.default_rng(1).normal(size=nx * ny * nz)
    g = 0.0123
    xs = [m.solve_shifted(g, b, method=meth) for meth in (O.SOLVE_DCT, O.SOLVE_CG, O.SOLVE_DENSE)]
    for x in xs:
        assert np.abs(x - g * m.laplacian(x) - b).max() < 1e-13 * np.abs(b).max()
    np.testing.assert_allclose(xs[0], xs[2], atol=1e-13)
    np.testing.assert_allclose(xs[1], xs[2], atol=1e-13)


@pytest.mark.parametrize("shape", [(6, 5, 1), (5, 4, 3)])
def test_field_spectrum_inside_gershgorin_interval(orc, shape):
    # The interval of the Chebyshev solves for a conductivity field: 1 is the
    # smallest eigenvalue of I - g A (constants), and twice the largest
    # diagonal of -A, max_p sum_faces (sigma_p + sigma_q)/h^2, bounds the rest.
    nx, ny, nz = shape
    h, g = 0.3, 0.2
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.h = h
    wl.sigma_field = I.lognormal_field(nx, ny, nz, seed=11, corr=2.0)
    m = O.Monodomain(wl, solver=O.SOLVE_CG)
    N = nx * ny * nz
    B = np.stack([e - g * m.conductivity(e) for e in np.eye(N)], axis=1)
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    sg = wl.sigma_field.reshape(nz, ny, nx)
    G = 0.0
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                s = 0.0
                for dz, dy, dx in ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
                    jz, jy, jx = iz + dz, iy + dy, ix + dx
                    if 0 <= jz < nz and 0 <= jy < ny and 0 <= jx < nx:
                        s += sg[iz, iy, ix] + sg[jz, jy, jx]
                G = max(G, s / h**2)
    assert abs(ev.min() - 1.0) < 1e-12
    assert ev.max() <= 1 + g * G + 1e-12
    assert ev.max() >= 1 + 0.5 * g * G


@pytest.mark.parametrize("shape", [(7, 1, 1), (6, 5, 1), (5, 4, 3), (2, 3, 2)])
def test_laplacian4_spectrum_interval(orc, shape):
    # The fourth-order operator's spectrum: I - g L4 fills exactly
    # [1, 1 + (g/(12 h^2)) sum_axes (30 + 2 cos 2t - 32 cos t)], t = pi (n-1)/n.
    nx, ny, nz = shape
    h, g = 0.3, 0.05
    wl = I.hh_sheet_32().with_mesh(nx, ny, nz)
    wl.h = h
    wl.order = 4
    m = O.Monodomain(wl)
    N = nx * ny * nz
    B = np.stack([e - g * m.laplacian(e) for e in np.eye(N)], axis=1)
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    hi = 1 + g / (12 * h**2) * sum(30 + 2 * np.cos(2 * np.pi * (n - 1) / n) - 32 * np.cos(np.pi * (n - 1) / n)
                                   for n in shape if n > 1)
    assert abs(ev.min() - 1.0) < 1e-12 and abs(ev.max() - hi) < 1e-12 * hi
