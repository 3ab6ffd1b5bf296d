"""Pins of the oracle's particle mover (Eqs. 3, 13-16 and the RK4 reading A1).

Closed forms used: special-relativistic gyration in a uniform B (m = 0), Schwarzschild and
Bardeen-Press-Teukolsky circular orbits, conservation of -u_4, u_phi and g(u,u) along
geodesics, and the convergence order of RK4.
"""
import numpy as np
import pytest

import oracle as O


def _test_particle_run(N, m, a, dt, x_rel, u, nsteps, B=(0.0, 0.0, 0.0), E=(0.0, 0.0, 0.0), qm=0.0, c=1.0,
                       flags=0):
    o = O.Oracle(N, N, N, m, a, c, dt, flags=O.FROZEN_FIELDS | flags, threads=1)
    o.init_uniform_field(E=E, B=B)
    Xc = o.centre
    x4 = np.array([[Xc[0] + x_rel[0]], [Xc[1] + x_rel[1]], [Xc[2] + x_rel[2]], [0.0]])
    o.load_particles(0, qm, 0.0, x4, np.asarray(u, float).reshape(4, 1), [7])
    traj = []
    for _ in range(nsteps):
        o.step(1)
        x, uu, _ = o.get_particles(0)
        traj.append((x[:, 0] - np.r_[Xc, 0.0], uu[:, 0]))
    return traj


def _gyration_error(dt, flags=0):
    """m = 0, uniform contravariant B_z, E = 0: u_perp rotates at (q/m) B per unit proper time."""
    c, qm, B0, u0 = 1.0, 1.0, 0.5, 0.6
    u4 = c * np.sqrt(1 + (u0 / c) ** 2)
    T = 6.0
    n = int(round(T / dt))
    traj = _test_particle_run(24, 0.0, 0.0, dt, (0.0, 0.0, 0.0), (u0, 0.0, 0.0, u4), n, B=(0, 0, B0), qm=qm,
                              flags=flags)
    x, u = traj[-1]
    tau = n * dt / (u4 / c)
    w = qm * B0
    u_ref = np.array([u0 * np.cos(w * tau), -u0 * np.sin(w * tau), 0.0, u4])
    x_ref = np.array([u0 / w * np.sin(w * tau), u0 / w * (np.cos(w * tau) - 1), 0.0, c * n * dt])
    return np.abs(u - u_ref).max(), np.abs(x - x_ref).max()


def test_flat_gyration_closed_form_and_order():
    e1u, e1x = _gyration_error(0.4)
    e2u, e2x = _gyration_error(0.2)
    assert e1u < 1e-4 and e1x < 1e-3
    order_u = np.log2(e1u / e2u)
    order_x = np.log2(e1x / e2x)
    assert 3.8 < order_u < 4.2, order_u
    assert 3.8 < order_x < 4.2, order_x


def test_rk4_as_printed_ablation():
    """The RK4 steps of Sec. 3.3 as printed (finals taken as increments of x_n and u_n; oracle
    switch RK4_AS_PRINTED).  With m = 0, E = 0 and a uniform B_z nothing changes u^4, so every
    gamma_k of Eq. 16 is u^4/c and the printed stage steps dt/(2 gamma), dt/gamma, dt/gamma,
    dt/(2 gamma) weighted 1, 2, 2, 1 over 6 advance proper time by 5/6 of dt/gamma: x^4 gains
    5/6 c dt per step, and the gyration phase lags by a fixed fraction that no step size
    removes (an inconsistent scheme).  The classical reading (A1) converges at fourth order
    (test_flat_gyration_closed_form_and_order)."""
    c, dt, u0 = 1.0, 0.4, 0.6
    u4 = c * np.sqrt(1 + u0 ** 2)
    traj = _test_particle_run(24, 0.0, 0.0, dt, (0.0, 0.0, 0.0), (u0, 0.0, 0.0, u4), 5, B=(0, 0, 0.5), qm=1.0,
                              flags=O.RK4_AS_PRINTED)
    for k, (x, u) in enumerate(traj, start=1):
        assert x[3] == pytest.approx(k * 5.0 / 6.0 * c * dt, rel=1e-14)
        assert u[3] == pytest.approx(u4, rel=1e-14)
    e1u, _ = _gyration_error(0.4, O.RK4_AS_PRINTED)
    e2u, _ = _gyration_error(0.2, O.RK4_AS_PRINTED)
    c1u, _ = _gyration_error(0.4)
    assert e1u > 1e3 * c1u
    assert e2u > 0.5 * e1u  # halving dt does not shrink the error


def test_lorentz_force_flat():
    """m = 0: a~ = (q/m)(gamma c E + u x B) spatially and (q/m) E.u for the time part."""
    c, qm = 1.0, -0.7
    E = np.array([0.01, -0.02, 0.015])
    B = np.array([0.05, 0.02, -0.1])
    o = O.Oracle(16, 16, 16, 0.0, 0.0, c, 0.4, flags=O.FROZEN_FIELDS)
    o.init_uniform_field(E=E, B=B)
    usp = np.array([0.3, -0.2, 0.5])
    u = np.r_[usp, c * np.sqrt(1 + usp @ usp / c**2)]
    x = np.array([7.3, 8.1, 6.6, 0.0])
    acc = o.accel(qm, x, u)
    ref_sp = qm * (u[3] / c * c * E + np.cross(usp, B))
    ref_t = qm * (E @ usp)
    assert np.allclose(acc[:3], ref_sp, rtol=1e-13, atol=1e-16)
    assert acc[3] == pytest.approx(ref_t, rel=1e-13)


def test_schwarzschild_circular_orbit():
    """a = 0 circular geodesic at r = 6.5m: dphi/dt = sqrt(m/r^3), u^4/c = 1/sqrt(1 - 3m/r)."""
    m, r, dt, c = 1.0, 6.5, 0.25, 1.0
    u4 = c / np.sqrt(1 - 3 * m / r)
    Om = np.sqrt(m / r**3)
    n = 300
    traj = _test_particle_run(22, m, 0.0, dt, (r, 0.0, 0.0), (0.0, r * Om * u4, 0.0, u4), n)
    for x, u in traj[::30]:
        t = x[3] / c
        assert np.hypot(x[0], x[1]) == pytest.approx(r, rel=2e-6)
        assert np.arctan2(x[1], x[0]) % (2 * np.pi) == pytest.approx((Om * t) % (2 * np.pi), abs=2e-5)
        assert u[3] == pytest.approx(u4, rel=1e-6)


def test_kerr_equatorial_circular_orbits():
    """Bardeen-Press-Teukolsky: dphi/dt = +-sqrt(m)/(r^1.5 +- a sqrt(m)) for prograde (+) and
    retrograde (-) orbits; with the paper's sign in Eq. 5 the hole drags towards -phi."""
    m, a, r, dt, c = 1.0, 0.9, 7.0, 0.25, 1.0
    R = np.sqrt(r * r + a * a)
    X = np.array([R, 0.0, 0.0])
    drag = -np.sign(np.array([0, 0, 0, 1.0]) @ O.metric(X, m, a) @ np.array([0.0, R, 0, 0]))
    assert drag < 0
    for prograde in (True, False):
        Om = np.sqrt(m) / (r**1.5 + (a if prograde else -a) * np.sqrt(m))
        Om *= drag if prograde else -drag
        v = np.array([0.0, R * Om, 0.0])
        gam = O.gamma_from_v(X, m, a, c, v)
        u = np.r_[gam * v, gam * c]
        traj = _test_particle_run(22, m, a, dt, X, u, 200)
        for x, uu in traj[::20]:
            t = x[3] / c
            assert np.hypot(x[0], x[1]) == pytest.approx(R, rel=5e-6)
            dphi = (np.arctan2(x[1], x[0]) - Om * t + np.pi) % (2 * np.pi) - np.pi
            assert abs(dphi) < 5e-5


def _invariants(x, u, m, a, c):
    g = O.metric(x[:3], m, a)
    ul = g @ u
    return np.array([u @ g @ u + c * c, -ul[3], -x[1] * ul[0] + x[0] * ul[1]])


def _geodesic_drift(dt, m=1.0, a=0.7, c=1.0):
    X = np.array([7.0, 0.5, 1.2])
    usp = np.array([0.03, 0.36, 0.05])  # contravariant u^i: a bound, eccentric, inclined orbit
    u = O.solve_u4(X, m, a, c, usp, 2)
    T = 40.0
    n = int(round(T / dt))
    traj = _test_particle_run(28, m, a, dt, X, u, n)
    I0 = _invariants(np.r_[X, 0.0], u, m, a, c)
    x, uu = traj[-1]
    return np.abs(_invariants(x, uu, m, a, c) - I0)


def test_geodesic_invariants_converge_fourth_order():
    """Killing energy -u_4, axial u_phi and the norm are conserved up to O(h^4)."""
    d1 = _geodesic_drift(0.4)
    d2 = _geodesic_drift(0.2)
    assert d1.max() < 1e-4
    for k in range(3):
        assert np.log2(d1[k] / d2[k]) > 3.5, (k, d1, d2)
