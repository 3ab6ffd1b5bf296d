"""Pins of the oracle's staggered gather and of the charged push in a non-uniform field.

Sec. 3.3 interpolates each field component to the particle with sqrt(-g)-weighted cell
sub-volumes; with det g = -1 (reading A5) these are trilinear weights about the component's own
Yee lattice (Sec. 3, Fig. 2): d^x at (i+1/2, j, k), d^y at (i, j+1/2, k), d^z at (i, j, k+1/2),
b_x at (i, j+1/2, k+1/2), b_y at (i+1/2, j, k+1/2), b_z at (i+1/2, j+1/2, k).  Trilinear
interpolation reproduces an affine function exactly, so a field that is affine in position with
a different gradient per component is gathered exactly at any point -- and a wrong half-cell
offset or swapped weights shift the result by half a gradient.

Eq. 15 with a field that is not uniform: Wald's stationary vacuum field
A = (B0/2)(xi_phi + 2 a xi_t) is built from the two Killing vectors of the Kerr metric, so for a
charge the momenta -(u_4 + (q/m) A_4) and u_phi + (q/m) A_phi are conserved along its orbit; the
RK4 push (reading A1) keeps them to O(h^4).
"""
import numpy as np
import pytest

import oracle as O

# Yee offsets of the six prognostic components in half cells (Sec. 3, Fig. 2)
YEE = {0: (1, 0, 0), 1: (0, 1, 0), 2: (0, 0, 1), 3: (0, 1, 1), 4: (1, 0, 1), 5: (1, 1, 0)}


def _affine_fields(n, rng):
    """Per component c: value alpha_c + beta_c . (node position of its own lattice)."""
    alpha = rng.uniform(-1, 1, 6)
    beta = rng.uniform(-0.2, 0.2, (6, 3))
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    F = np.zeros((6, n, n, n))
    for c in range(6):
        off = 0.5 * np.array(YEE[c])
        F[c] = alpha[c] + beta[c, 0] * (i + off[0]) + beta[c, 1] * (j + off[1]) + beta[c, 2] * (k + off[2])
    return alpha, beta, F


def _value(alpha, beta, c, x):
    return alpha[c] + beta[c] @ x


@pytest.mark.parametrize("m,a", [(0.0, 0.0), (2.0, 0.9)])
def test_gather_reproduces_affine_fields(m, a):
    n = 14
    rng = np.random.default_rng(11)
    alpha, beta, F = _affine_fields(n, rng)
    o = O.Oracle(n, n, n, m, a, 1.0, 0.4, flags=O.FROZEN_FIELDS)
    o.set_fields(F[:3], F[3:])
    for x in rng.uniform(1.0, n - 2.0, (200, 3)):
        for c in range(6):
            assert o.gather(c, x) == pytest.approx(_value(alpha, beta, c, x), rel=1e-13, abs=1e-14)


def test_gather_is_not_the_node_lattice():
    """The same affine values placed on the wrong lattice would be gathered off by half a gradient:
    this checks that the comparison above can fail (each component's offset matters)."""
    n = 12
    rng = np.random.default_rng(3)
    alpha, beta, F = _affine_fields(n, rng)
    o = O.Oracle(n, n, n, 0.0, 0.0, 1.0, 0.4, flags=O.FROZEN_FIELDS)
    o.set_fields(F[:3], F[3:])
    x = np.array([5.3, 6.1, 4.7])
    for c in range(6):
        shifted = _value(alpha, beta, c, x + 0.5 * np.array(YEE[c]))  # as if stored at integer nodes
        if np.any(YEE[c]):
            assert abs(o.gather(c, x) - shifted) > 1e-3


def test_accel_flat_affine_field_closed_form():
    """m = 0: a~ = (q/m)(gamma c E + u x B) and (q/m) E.u with E = -d(x), B = b(x) at the particle."""
    n, c, qm = 14, 1.0, -0.8
    rng = np.random.default_rng(5)
    alpha, beta, F = _affine_fields(n, rng)
    o = O.Oracle(n, n, n, 0.0, 0.0, c, 0.4, flags=O.FROZEN_FIELDS)
    o.set_fields(F[:3], F[3:])
    for x in rng.uniform(1.5, n - 2.5, (40, 3)):
        E = -np.array([_value(alpha, beta, q, x) for q in range(3)])
        B = np.array([_value(alpha, beta, 3 + q, x) for q in range(3)])
        usp = rng.normal(0, 0.4, 3)
        u = np.r_[usp, c * np.sqrt(1 + usp @ usp / c**2)]
        acc = o.accel(qm, np.r_[x, 0.0], u)
        assert np.allclose(acc[:3], qm * (u[3] * E + np.cross(usp, B)), rtol=1e-12, atol=1e-14)
        assert acc[3] == pytest.approx(qm * (E @ usp), rel=1e-12, abs=1e-14)


def test_accel_curved_affine_field():
    """m > 0: a~ = (q/m) F^a_c g_cb u^b - Gamma^a_mn u^m u^n with F completed at the particle from the
    affine (b, d) there (the completion and Gamma are pinned in test_oracle_fields/metric)."""
    n, m, a, c, qm = 16, 2.0, 0.9, 1.0, 0.6
    rng = np.random.default_rng(9)
    alpha, beta, F = _affine_fields(n, rng)
    o = O.Oracle(n, n, n, m, a, c, 0.4, flags=O.FROZEN_FIELDS)
    o.set_fields(F[:3], F[3:])
    Xc = np.array(o.centre)
    for x in rng.uniform(1.5, n - 2.5, (40, 3)):
        X = x - Xc
        if np.linalg.norm(X) < 2.5 * m:
            continue
        g = O.metric(X, m, a)
        d = np.array([_value(alpha, beta, q, x) for q in range(3)])
        b = np.array([_value(alpha, beta, 3 + q, x) for q in range(3)])
        Fu, _ = O.complete_tensor(g, b, d)
        G = O.christoffel(X, m, a)
        usp = rng.normal(0, 0.3, 3)
        u = O.solve_u4(X, m, a, c, usp, 2)
        ref = qm * (Fu @ g @ u) - np.einsum("amn,m,n->a", G, u, u)
        acc = o.accel(qm, np.r_[x, 0.0], u)
        assert np.allclose(acc, ref, rtol=1e-11, atol=1e-13)


def _wald_momenta(x, u, m, a, c, qm, B0):
    X = x[:3]
    g = O.metric(X, m, a)
    xi = np.array([-X[1], X[0], 0.0, 2.0 * a])
    A = 0.5 * B0 * (g @ xi)  # A_mu = (B0/2) g_mu nu (xi_phi + 2 a xi_t)^nu
    ul = g @ u
    energy = -(ul[3] + qm * A[3])
    ang = (-X[1] * ul[0] + X[0] * ul[1]) + qm * (-X[1] * A[0] + X[0] * A[1])
    return np.array([energy, ang, u @ g @ u + c * c])


def _wald_drift(dt, qm, m=1.0, a=0.7, c=1.0, B0=0.25):
    N = 32
    o = O.Oracle(N, N, N, m, a, c, dt, flags=O.FROZEN_FIELDS | O.ANALYTIC_WALD, threads=1)
    o.set_wald_b0(B0)
    Xc = np.array(o.centre)
    X = np.array([7.0, 0.5, 1.2])
    # azimuthal velocity against the magnetic force's sense, so that the orbit stays bound outside r = 7m
    u = O.solve_u4(X, m, a, c, np.array([0.05, 0.3 * np.sign(qm), 0.08]), 2)
    o.load_particles(0, qm, 0.0, np.r_[Xc + X, 0.0].reshape(4, 1), u.reshape(4, 1), [1])
    I0 = _wald_momenta(np.r_[X, 0.0], u, m, a, c, qm, B0)
    n = int(round(30.0 / dt))
    rmin = 1e9
    for _ in range(n):
        o.push_deposit()
        xx, uu, _ = o.get_particles(0)
        rmin = min(rmin, np.linalg.norm(xx[:3, 0] - Xc))
    x1 = np.r_[xx[:3, 0] - Xc, 0.0]
    return np.abs(_wald_momenta(x1, uu[:, 0], m, a, c, qm, B0) - I0), rmin


@pytest.mark.parametrize("qm", [0.5, -0.5])
def test_charged_orbit_in_wald_field_conserves_momenta_fourth_order(qm):
    d1, r1 = _wald_drift(0.4, qm)
    d2, _ = _wald_drift(0.2, qm)
    assert r1 > 3.0  # the orbit stays well outside the horizon
    assert d1.max() < 1e-3, d1
    for k in range(3):
        assert np.log2(d1[k] / d2[k]) > 3.5, (k, d1, d2)


def test_wald_momenta_are_not_trivially_conserved():
    """Without the (q/m) A terms the kinetic -u_4 and u_phi change along the charged orbit by far more
    than the drift bound above (the field does work on the particle)."""
    m, a, c, qm, B0, dt = 1.0, 0.7, 1.0, 0.5, 0.25, 0.4
    N = 32
    o = O.Oracle(N, N, N, m, a, c, dt, flags=O.FROZEN_FIELDS | O.ANALYTIC_WALD, threads=1)
    o.set_wald_b0(B0)
    Xc = np.array(o.centre)
    X = np.array([7.0, 0.5, 1.2])
    u = O.solve_u4(X, m, a, c, np.array([0.05, 0.3, 0.08]), 2)
    o.load_particles(0, qm, 0.0, np.r_[Xc + X, 0.0].reshape(4, 1), u.reshape(4, 1), [1])
    k0 = _wald_momenta(np.r_[X, 0.0], u, m, a, c, 0.0, B0)
    for _ in range(75):
        o.push_deposit()
    xx, uu, _ = o.get_particles(0)
    k1 = _wald_momenta(np.r_[xx[:3, 0] - Xc, 0.0], uu[:, 0], m, a, c, 0.0, B0)
    assert abs(k1[1] - k0[1]) > 1e-2
