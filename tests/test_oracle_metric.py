"""Pins of the oracle's metric module (Eqs. 4-7, 16) against what the mathematics fixes.

Boyer-Lindquist invariants are used where possible: g(d_t, d_t), g(d_t, d_phi), g(d_phi, d_phi)
and g^{mn} d_m r d_n r do not depend on the coordinates, so they pin Eqs. 4-6 (and the
numerical inverse) without retyping them.
"""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(12345)
CASES = [(2.0, 0.0), (1.0, 0.5), (4.0, 3.6), (3.0, 2.97), (8.0, 7.6)]


def _points(m, n=25):
    pts = []
    while len(pts) < n:
        X = RNG.uniform(-6 * m - 3, 6 * m + 3, 3)
        if np.linalg.norm(X) > 1.2 * m + 1.0:
            pts.append(X)
    return pts


@pytest.mark.parametrize("m,a", CASES)
def test_quartic_root(m, a):
    """Eq. 6: r is the non-negative root; special cases on the axis, in the equator, a = 0."""
    for X in _points(m):
        r = O.kerr_r(X, a)
        R2 = X @ X
        res = r**4 - (R2 - a * a) * r * r - a * a * X[2] ** 2
        assert abs(res) <= 1e-13 * max(1.0, R2 * R2)
        assert r >= 0
        if a == 0:
            assert r == pytest.approx(np.sqrt(R2), rel=1e-15)
    for z in (0.3, 2.0, -7.5):
        assert O.kerr_r(np.array([0.0, 0.0, z]), a) == pytest.approx(abs(z), rel=1e-14)
    for R in (a + 0.5, 2 * a + 3, 10.0):
        X = np.array([R / np.sqrt(2), R / np.sqrt(2), 0.0])
        assert O.kerr_r(X, a) == pytest.approx(np.sqrt(R * R - a * a), rel=1e-14)


@pytest.mark.parametrize("m,a", CASES)
def test_null_vector_and_determinant(m, a):
    """k is null for eta (follows from Eq. 6), so det g = -1 and g^{-1} = eta - f k^ k^."""
    eta = np.diag([1.0, 1.0, 1.0, -1.0])
    for X in _points(m):
        r, f, k = O.kerr_fk(X, m, a)
        assert abs(k @ eta @ k) < 1e-14
        assert O.metric_det(X, m, a) == pytest.approx(-1.0, abs=1e-13)
        g = O.metric(X, m, a)
        gi = O.metric_inverse(X, m, a)
        assert np.abs(g @ gi - np.eye(4)).max() < 1e-13
        assert np.abs(g - g.T).max() < 1e-15 * np.abs(g).max()


def _bl(X, m, a):
    r = O.kerr_r(X, a)
    cos_t = X[2] / r
    sin2 = 1.0 - cos_t**2
    Sigma = r * r + a * a * cos_t**2
    Delta = r * r - 2 * m * r + a * a
    return r, sin2, Sigma, Delta


@pytest.mark.parametrize("m,a", CASES)
def test_boyer_lindquist_invariants(m, a):
    """g(d_t,d_t) = -(1 - 2mr/Sigma), |g(d_t,d_phi)| = 2 m a r sin^2/Sigma,
    g(d_phi,d_phi) = (r^2 + a^2 + 2 m a^2 r sin^2/Sigma) sin^2, g^{mn} r_m r_n = Delta/Sigma."""
    for X in _points(m):
        r, sin2, Sigma, Delta = _bl(X, m, a)
        g = O.metric(X, m, a)
        gi = O.metric_inverse(X, m, a)
        xi_phi = np.array([-X[1], X[0], 0.0, 0.0])
        xi_t = np.array([0.0, 0.0, 0.0, 1.0])
        assert xi_t @ g @ xi_t == pytest.approx(-(1 - 2 * m * r / Sigma), abs=1e-13)
        assert abs(xi_t @ g @ xi_phi) == pytest.approx(2 * m * a * r * sin2 / Sigma, abs=1e-12)
        gpp = (r * r + a * a + 2 * m * a * a * r * sin2 / Sigma) * sin2
        assert xi_phi @ g @ xi_phi == pytest.approx(gpp, rel=1e-12, abs=1e-12)
        # gradient of r by centred differences of the root itself (independent of Eq. 4)
        h = 1e-5
        dr = np.zeros(4)
        for l in range(3):
            e = np.zeros(3)
            e[l] = h
            dr[l] = (O.kerr_r(X + e, a) - O.kerr_r(X - e, a)) / (2 * h)
        assert dr @ gi @ dr == pytest.approx(Delta / Sigma, rel=1e-8, abs=1e-9)


def test_horizon_is_null_surface():
    """At r = r_+ = m + sqrt(m^2 - a^2) the surface r = const is null (Delta = 0)."""
    m, a = 4.0, 3.6
    rp = m + np.sqrt(m * m - a * a)
    for th in (0.3, 1.0, 1.5707963):
        # a point with BL radius rp: x^2 + y^2 = (rp^2 + a^2) sin^2, z = rp cos
        X = np.array([np.sqrt(rp * rp + a * a) * np.sin(th), 0.0, rp * np.cos(th)])
        assert O.kerr_r(X, a) == pytest.approx(rp, rel=1e-13)
        r, sin2, Sigma, Delta = _bl(X, m, a)
        assert abs(Delta) < 1e-12


@pytest.mark.parametrize("m,a", CASES)
def test_christoffel_against_finite_differences(m, a):
    """Dual-number Gamma vs Gamma from Richardson-extrapolated centred differences of g."""
    for X in _points(m, 8):
        G = O.christoffel(X, m, a)
        gi = O.metric_inverse(X, m, a)
        dg = np.zeros((4, 4, 4))

        def cd(h, l):
            e = np.zeros(3)
            e[l] = h
            return (O.metric(X + e, m, a) - O.metric(X - e, m, a)) / (2 * h)

        for l in range(3):
            h = 1e-3
            dg[l] = (4 * cd(h / 2, l) - cd(h, l)) / 3
        Gfd = 0.5 * (np.einsum("ab,mbn->amn", gi, dg) + np.einsum("ab,nbm->amn", gi, dg)
                     - np.einsum("ab,bmn->amn", gi, dg))
        scale = max(1.0, np.abs(G).max())
        assert np.abs(G - Gfd).max() < 1e-8 * scale
        assert np.abs(G - G.transpose(0, 2, 1)).max() < 1e-15 * scale


def test_gauss_legendre_matches_library():
    """Nodes/weights equal numpy's Golub-Welsch values; exact on degree 2Q-1."""
    for Q in range(1, 9):
        x, w = O.gauss_legendre(Q)
        xr, wr = np.polynomial.legendre.leggauss(Q)
        assert np.allclose(x, xr, atol=1e-14) and np.allclose(w, wr, atol=1e-14)
        for deg in range(2 * Q):
            exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
            assert (w * x**deg).sum() == pytest.approx(exact, abs=1e-13)


@pytest.mark.parametrize("m,a", CASES)
def test_solve_u4_and_eq7(m, a):
    """Completed 4-velocities are unit, future-directed, and Eq. 7 gives gamma = u^4/c."""
    c = 1.0
    for X in _points(m, 10):
        usp = RNG.normal(0, 0.3, 3)
        u = O.solve_u4(X, m, a, c, usp, 1)
        g = O.metric(X, m, a)
        assert u @ g @ u == pytest.approx(-c * c, abs=1e-13)
        assert u[3] > 0
        ul = g @ u
        assert np.allclose(ul[:3], usp, atol=1e-14)
        if g[3, 3] < 0:
            u2 = O.solve_u4(X, m, a, c, u[:3], 2)
            assert np.allclose(u2, u, rtol=1e-12, atol=1e-14)
        v = u[:3] / (u[3] / c)
        assert O.gamma_from_v(X, m, a, c, v) == pytest.approx(u[3] / c, rel=1e-12)


def test_gamma_function_eq16():
    """Eq. 16 solves c dt = u^4 dtau + a^4 dtau^2 / 2 with dtau = dt / gamma."""
    c, dt = 1.0, 0.4
    for u4, a4 in [(1.0, 0.0), (1.3, 0.2), (2.0, -0.7), (1.05, 0.01)]:
        g, fb = O.gamma_f(u4, a4, c, dt)
        assert not fb
        dtau = dt / g
        assert u4 * dtau + 0.5 * a4 * dtau**2 == pytest.approx(c * dt, rel=1e-14)
    g, fb = O.gamma_f(1.2, 0.0, c, dt)
    assert g == pytest.approx(1.2, rel=1e-15)
    g, fb = O.gamma_f(1.0, -10.0, c, dt)  # negative argument: reading A2 fallback
    assert fb and g == 1.0


@pytest.mark.parametrize("m,a", [(2.0, 0.0), (4.0, 3.6)])
def test_volume_weights_are_trilinear(m, a):
    """Sec. 3.3: sub-volumes of sqrt(-det g) give exactly trilinear CIC weights (det g = -1)."""
    Xc = np.array([15.5, 15.5, 15.5])
    for _ in range(5):
        cell = RNG.integers(18, 25, 3)
        w = RNG.uniform(0, 1, 3)
        P = cell + w
        W = O.volume_weights(P, cell, Xc, m, a, 2)
        wx, wy, wz = w
        tri = [(1 - wx) * (1 - wy) * (1 - wz), wx * (1 - wy) * (1 - wz), (1 - wx) * wy * (1 - wz),
               (1 - wx) * (1 - wy) * wz, wx * wy * (1 - wz), (1 - wx) * wy * wz, wx * (1 - wy) * wz,
               wx * wy * wz]
        assert np.allclose(W, tri, atol=1e-14)
