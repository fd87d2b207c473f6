"""Pins of the oracle's collocation data against closed forms and independent
library routes (Sec. 3.1.2 Radau IIA nodes; eq. def_aij; App. A eqs. fornberg,
def_aij_computable, def_phik).  The paper prints no numbers for these, so each
pin is a textbook closed form, an exact identity, or a high-precision mpmath
evaluation of the defining integral."""
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("M", [2, 3])
def test_radau_nodes_closed_form(orc, M):
    # Radau IIA right nodes: M=2 -> {1/3, 1}; M=3 -> {(4-sqrt6)/10, (4+sqrt6)/10, 1}
    c = O.radau_nodes(M)
    want = {2: [0, 1 / 3, 1], 3: [0, (4 - math.sqrt(6)) / 10, (4 + math.sqrt(6)) / 10, 1]}[M]
    np.testing.assert_allclose(c, want, rtol=0, atol=2e-16)


@pytest.mark.parametrize("M", range(1, 9))
def test_radau_quadrature_degree(orc, M):
    # The last row of q is the Radau quadrature: exact for degree <= 2M-2, not for 2M-1.
    c = O.radau_nodes(M)[1:]
    b = O.collocation_q(M)[-1]
    for m in range(0, 2 * M - 1):
        assert abs(b @ c**m - 1.0 / (m + 1)) < 5e-15, (M, m)
    assert abs(b @ c ** (2 * M - 1) - 1.0 / (2 * M)) > 1e-12   # not exact one degree higher
    assert abs(b.sum() - 1.0) < 5e-15


def test_radau_iia_m3_matrix_textbook(orc):
    # Closed-form Radau IIA coefficients (3 stages, order 5), the standard
    # table of Hairer & Wanner, Solving ODEs II, Sec. IV.5.
    s6 = math.sqrt(6.0)
    A = np.array([[(88 - 7 * s6) / 360, (296 - 169 * s6) / 1800, (-2 + 3 * s6) / 225],
                  [(296 + 169 * s6) / 1800, (88 + 7 * s6) / 360, (-2 - 3 * s6) / 225],
                  [(16 - s6) / 36, (16 + s6) / 36, 1 / 9]])
    np.testing.assert_allclose(O.collocation_q(3), A, rtol=0, atol=3e-16)


@pytest.mark.parametrize("M", range(1, 9))
def test_collocation_conditions(orc, M):
    # C(q): sum_j q_ij c_j^m = c_i^{m+1}/(m+1), m = 0..M-1
    c = O.radau_nodes(M)[1:]
    q = O.collocation_q(M)
    for m in range(M):
        np.testing.assert_allclose(q @ c**m, c ** (m + 1) / (m + 1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("M", range(1, 9))
def test_fornberg_matches_vandermonde_inverse(orc, M):
    # p(s) = sum_m a_m s^m, V a = p(c)  =>  p^{(k)}(0) = k! (V^{-1} p(c))_k
    c = O.radau_nodes(M)[1:]
    V = np.vander(c, M, increasing=True)
    want = np.array([math.factorial(k) for k in range(M)])[:, None] * np.linalg.inv(V)
    w = O.fornberg_weights(M)
    np.testing.assert_allclose(w, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    # exactness on monomials: sum_l w^k_l c_l^m = k! delta_km
    for k in range(M):
        for m in range(M):
            assert abs(w[k] @ c**m - (math.factorial(k) if k == m else 0.0)) < 1e-10 * max(1, np.abs(w[k]).sum())


def _phi_mp(k, z):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 160   # the closed form cancels ~k*log10(1/|z|) digits for tiny z
    z = mp.mpf(z)
    if z == 0:
        return 1.0 / math.factorial(k)
    s = mp.exp(z) - sum(z**m / mp.factorial(m) for m in range(k))
    return float(s / z**k)


ZS = [0.0, -1e-12, -1e-8, -1e-3, -0.3, -1.0, -1.999, -2.0, -2.001, -3.7, -10.0, -55.5,
      -100.0, -333.3, -500.0, -2000.0, 0.5, 1.9]


@pytest.mark.parametrize("z", ZS)
def test_phi_closed_form(orc, z):
    # phi_k(z) = (e^z - sum_{m<k} z^m/m!) / z^k, evaluated at 160 digits
    ph = O.phi(z, 8)
    for k in range(1, 9):
        want = _phi_mp(k, z)
        assert abs(ph[k - 1] - want) <= 4e-15 * abs(want), (k, z, ph[k - 1], want)


# The formula of App. A sums c_i^k w_j^{k-1} phi_k with Fornberg weights that
# grow quickly with M (max |w| ~ 1e2 at M=4, 1e7 at M=8), so its rounding error
# grows with M.  Tolerances below follow that growth.
AIJ_TOL = {1: 2e-15, 2: 2e-15, 3: 2e-15, 4: 5e-15, 5: 1e-14, 6: 5e-14, 7: 3e-13, 8: 1e-12}


@pytest.mark.parametrize("M", range(1, 9))
def test_aij_zero_is_collocation_matrix(orc, M):
    # a_ij(0) = q_ij (Sec. 3.1.2: standard collocation weights); two independent routes
    np.testing.assert_allclose(O.aij(M, 0.0), O.collocation_q(M), rtol=0, atol=AIJ_TOL[M])


@pytest.mark.parametrize("M", [2, 3, 4, 6])
@pytest.mark.parametrize("z", [-1e-6, -0.4, -2.5, -37.0, -500.0])
def test_aij_moment_identities(orc, M, z):
    # l_j interpolates s^m exactly (m < M), so
    # sum_j a_ij(z) c_j^m = int_0^{c_i} e^{(c_i-s)z} s^m ds = m! c_i^{m+1} phi_{m+1}(c_i z)
    c = O.radau_nodes(M)[1:]
    a = O.aij(M, z)
    for m in range(M):
        for i in range(M):
            want = math.factorial(m) * c[i] ** (m + 1) * _phi_mp(m + 1, c[i] * z)
            got = a[i] @ c**m
            assert abs(got - want) <= 1e-13 * abs(want) + AIJ_TOL[M], (M, z, m, i, got, want)


@pytest.mark.parametrize("M", [3, 4])
@pytest.mark.parametrize("z", [-0.7, -6.0, -80.0])
def test_aij_direct_integral(orc, M, z):
    # eq. def_aij evaluated directly by mpmath quadrature of e^{(c_i-s)z} l_j(s)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    c = [mp.mpf(x) for x in O.radau_nodes(M)]
    a = O.aij(M, z)
    for i in range(1, M + 1):
        for j in range(1, M + 1):
            def lj(s, j=j):
                p = mp.mpf(1)
                for k in range(1, M + 1):
                    if k != j:
                        p *= (s - c[k]) / (c[j] - c[k])
                return p
            f = lambda s: mp.exp((c[i] - s) * z) * lj(s)
            pts = [0, c[i] - min(c[i], mp.mpf(1) / abs(z)), c[i]]
            want = float(mp.quad(f, sorted(set(pts))))
            assert abs(a[i - 1, j - 1] - want) <= AIJ_TOL[M], (i, j, a[i - 1, j - 1], want)


def test_gauss_legendre_rule(orc):
    x, w = O.gauss_legendre(16)
    ref_x, ref_w = np.polynomial.legendre.leggauss(16)
    np.testing.assert_allclose(np.sort(x), ref_x, atol=1e-15)
    np.testing.assert_allclose(w[np.argsort(x)], ref_w, atol=1e-15)
