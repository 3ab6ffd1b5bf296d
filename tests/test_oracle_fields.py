"""Pins of the oracle's field tensor handling and field advance (Eqs. 8-12, readings A6-A9).

* index lowering round trip of the field tensor against numpy's own contraction;
* m = 0: the scheme is exactly Yee -- a vacuum plane wave follows the closed-form discrete
  solution with the Yee dispersion relation to roundoff;
* m > 0: Wald's uniform-field solution satisfies Maxwell's equations in Kerr, and the
  one-step drift of the discrete scheme from it converges at second order;
* the Christoffel terms of Eq. 11 vanish (A6);
* Gauss's law (div E - 4 pi rho) is preserved by the full cycle with the charge-conserving
  deposit (pins the sign reading A8 against the deposit).
"""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(777)


def test_complete_tensor_roundtrip():
    """Given b = F_{yz,zx,xy} and d = F^{x4,y4,z4}, the full tensor is recovered."""
    for m, a in [(0.0, 0.0), (2.0, 1.5), (4.0, 3.9)]:
        for _ in range(10):
            X = RNG.uniform(-12, 12, 3)
            if np.linalg.norm(X) < 2.5 * m + 0.5:
                continue
            g = O.metric(X, m, a)
            A = RNG.normal(size=(4, 4))
            Fu = A - A.T
            Fd = np.einsum("ma,nb,ab->mn", g, g, Fu)
            b = np.array([Fd[1, 2], Fd[2, 0], Fd[0, 1]])
            d = Fu[:3, 3].copy()
            Fu2, Fd2 = O.complete_tensor(g, b, d)
            assert np.allclose(Fu2, Fu, atol=1e-12)
            assert np.allclose(Fd2, Fd, atol=1e-12)


def test_uniform_field_init():
    """Eq. 8 uniform contravariant field: d = F^{i4} = -E^i everywhere; b lowered with g."""
    N, m, a = 16, 2.0, 1.0
    E = np.array([0.01, 0.02, -0.03])
    B = np.array([0.0, 0.05, 0.1])
    o = O.Oracle(N, N, N, m, a, 1.0, 0.4)
    o.init_uniform_field(E=E, B=B)
    d, b, _ = o.get_fields()
    for q in range(3):
        assert np.all(d[q] == -E[q])
    Fu = np.zeros((4, 4))
    Fu[1, 2], Fu[2, 0], Fu[0, 1] = B
    Fu[:3, 3] = -E
    Fu = Fu - Fu.T
    Xc = o.centre
    for (i, j, k) in [(3, 4, 12), (10, 10, 5), (1, 14, 7)]:
        # b_z = F_xy lives at (i+1/2, j+1/2, k)
        X = np.array([i + 0.5, j + 0.5, k]) - Xc
        g = O.metric(X, m, a)
        Fd = g @ Fu @ g
        assert b[2, k, j, i] == pytest.approx(Fd[0, 1], rel=1e-13)


def _yee_fields(N, kx, ky, D, n, s):
    """Closed-form Yee mode with E along z: returns (d, b) at the start of step n
    (d at time n, b at time n - 1/2)."""
    w = 2 * np.arcsin(s * np.sqrt(np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2))
    Bx = -s * D * np.sin(ky / 2) / np.sin(w / 2)
    By = s * D * np.sin(kx / 2) / np.sin(w / 2)
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    d = np.zeros((3, N, N, N))
    b = np.zeros((3, N, N, N))
    d[2] = D * np.cos(kx * i + ky * j - w * n)
    b[0] = Bx * np.cos(kx * i + ky * (j + 0.5) - w * (n - 0.5))
    b[1] = By * np.cos(kx * (i + 0.5) + ky * j - w * (n - 0.5))
    return d, b


def test_flat_space_is_yee_plane_wave():
    """m = 0: one cycle (B/2, B/2, E) is Yee's scheme; sin^2(w/2) = s^2 sum sin^2(k_i/2)."""
    N, c, dt, nsteps = 32, 1.0, 0.5, 8
    s = c * dt
    kx, ky, D = 2 * np.pi * 3 / 29.0, 2 * np.pi * 2 / 31.0, 0.7
    o = O.Oracle(N, N, N, 0.0, 0.0, c, dt)
    d, b = _yee_fields(N, kx, ky, D, 0, s)
    o.set_fields(d, b)
    for n in range(1, nsteps + 1):
        o.b_half()
        o.b_half2()
        o.e_step()
        dn, bn, _ = o.get_fields()
        de, be = _yee_fields(N, kx, ky, D, n, s)
        lo, hi = nsteps + 3, N - nsteps - 3
        sl = (slice(None), slice(lo, hi), slice(lo, hi), slice(lo, hi))
        assert np.abs(dn[sl] - de[sl]).max() < 1e-13
        assert np.abs(bn[sl] - be[sl]).max() < 1e-13


def test_wald_field_solves_maxwell_in_kerr():
    """The oracle's Wald field obeys d_nu F^{mu nu} = 0 (sqrt(-g) = 1) and the Bianchi identity;
    this only holds if Eqs. 4-6 give a Ricci-flat metric and d_4, x d_y - y d_x are Killing."""
    m, a, B0 = 2.0, 1.6, 0.1
    h = 1e-4
    for X in [np.array([5.3, -3.1, 2.2]), np.array([-2.0, 6.0, -4.5]), np.array([8.0, 1.0, 0.5])]:
        scale = np.abs(O.wald_field(X, m, a, B0)[1]).max()
        div = np.zeros(4)
        bian = 0.0
        for nu in range(3):
            e = np.zeros(3)
            e[nu] = h
            Fp = O.wald_field(X + e, m, a, B0)
            Fm = O.wald_field(X - e, m, a, B0)
            div += (Fp[1][:, nu] - Fm[1][:, nu]) / (2 * h)
        dF = []
        for l in range(3):
            e = np.zeros(3)
            e[l] = h
            dF.append((O.wald_field(X + e, m, a, B0)[0] - O.wald_field(X - e, m, a, B0)[0]) / (2 * h))
        bian = dF[0][1, 2] + dF[1][2, 0] + dF[2][0, 1]
        assert np.abs(div).max() < 1e-9 * max(scale, 1e-3) / 1e-3
        assert abs(bian) < 1e-9


def _wald_one_step_drift(m, N):
    o = O.Oracle(N, N, N, m, 0.8 * m, 1.0, 0.4, threads=0, flags=O.NO_GAMMA_TERMS)
    o.init_wald(0.1)
    d0, b0, _ = o.get_fields()
    o.b_half()
    o.b_half2()
    o.e_step()
    d1, b1, _ = o.get_fields()
    Xc = (N - 1) / 2
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    R = np.sqrt((i - Xc) ** 2 + (j - Xc) ** 2 + (k - Xc) ** 2) / m
    inner = (i >= 2) & (i <= N - 3) & (j >= 2) & (j <= N - 3) & (k >= 2) & (k <= N - 3)
    out = []
    for lo, hi in [(2.5, 4.0), (4.0, 6.0)]:
        msk = (R >= lo) & (R < hi) & inner
        out.append(max(np.abs(d1 - d0).max(axis=0)[msk].max(), np.abs(b1 - b0).max(axis=0)[msk].max()))
    return np.array(out)


@pytest.mark.slow
def test_wald_drift_converges_second_order():
    """Doubling the resolution (m cells per unit mass, same dt in cells) cuts the one-step
    drift from the stationary Wald field by ~8 (2nd order in space x half the time step)."""
    d1 = _wald_one_step_drift(1.5, 24)
    d2 = _wald_one_step_drift(3.0, 48)
    ratio = d1 / d2
    assert np.all(ratio > 5.5), ratio
    assert d1.max() < 1e-2  # B0 = 0.1; coarse grid (1.5 cells per unit mass)


def test_e_step_christoffel_terms_vanish():
    """A6: Gamma^a_{cb} F^{cb} + Gamma^b_{bc} F^{ac} = 0 for this metric (sqrt(-g) = 1)."""
    N = 16
    o = O.Oracle(N, N, N, 2.0, 1.7, 1.0, 0.4)
    d = RNG.normal(size=(3, N, N, N)) * 0.1
    b = RNG.normal(size=(3, N, N, N)) * 0.1
    o.set_fields(d, b)
    o.e_step()
    gmax, gscale = o.gamma_terms()
    assert gscale > 1e-3
    assert gmax <= 1e-13 * gscale


def _div_E(d):
    E = -d
    div = np.zeros_like(E[0])
    div[:, :, 1:] += E[0][:, :, 1:] - E[0][:, :, :-1]
    div[:, 1:, :] += E[1][:, 1:, :] - E[1][:, :-1, :]
    div[1:, :, :] += E[2][1:, :, :] - E[2][:-1, :, :]
    return div


def test_gauss_law_flat_closed_form():
    """m = 0, gamma not applied to J (A13 off): over each full cycle, div E - 4 pi rho changes by
    exactly -4 pi times the deposit's closed-form 3-D continuity defect (zero for 2-D moves).
    This fixes the sign of J in the E step (A8) against the deposit and div curl = 0."""
    from test_oracle_deposit import cic_rho, cubic_defect

    N, c, dt, q = 20, 1.0, 0.4, 0.05
    o = O.Oracle(N, N, N, 0.0, 0.0, c, dt, flags=O.NO_GAMMA_IN_J)
    o.init_uniform_field(B=(0.0, 0.0, 0.2))
    n = 40
    x = np.vstack([RNG.uniform(8, 12, (3, n)), np.zeros((1, n))])
    usp = RNG.normal(0, 0.3, (3, n))
    u = np.vstack([usp, np.sqrt(1 + (usp**2).sum(0))])
    o.load_particles(0, -1.0, -q, x, u, np.arange(n))
    o.load_particles(1, 1.0, q, x + np.array([[0.3], [0.1], [-0.2], [0.0]]), u[[1, 0, 2, 3]], np.arange(n))
    sl = (slice(4, N - 4),) * 3
    charge = (-q, q)

    def gauss():
        d, _, _ = o.get_fields()
        rho = sum(cic_rho(N, o.get_particles(s)[0], charge[s]) for s in (0, 1))
        return _div_E(d) - 4 * np.pi * rho

    G = gauss()
    for _ in range(6):
        before = [o.get_particles(s)[0] for s in (0, 1)]
        o.step(1)
        after = [o.get_particles(s)[0] for s in (0, 1)]
        pred = np.zeros((N, N, N))
        for s in (0, 1):
            for p in range(n):
                pred += cubic_defect(N, before[s][:3, p], after[s][:3, p], charge[s])
        G1 = gauss()
        assert np.abs((G1 - G)[sl] + 4 * np.pi * pred[sl]).max() < 1e-14
        G = G1
    assert o.num_particles(0) == n and o.num_particles(1) == n



def test_contra_h_readout():
    """The contravariant read-out of the face components: in flat space h = b exactly; for the
    uniform contravariant field of Eq. 8 converted to b with the metric at every face, far from the
    hole (where g varies little over a cell) h returns B to within the averaging of neighbouring
    faces' b; the outer index layer reads zero."""
    N = 20
    flat = O.Oracle(N, N, N, 0.0, 0.0, 1.0, 0.4)
    rng = np.random.default_rng(4)
    d = rng.standard_normal((3, N, N, N))
    b = rng.standard_normal((3, N, N, N))
    flat.set_fields(d, b)
    h = flat.get_contra_h()
    assert np.array_equal(h[:, 1:-1, 1:-1, 1:-1], b[:, 1:-1, 1:-1, 1:-1])
    assert np.abs(h[:, 0]).max() == 0.0 and np.abs(h[:, :, :, -1]).max() == 0.0
    kerr = O.Oracle(N, N, N, 1.0, 0.9, 1.0, 0.4)
    B = np.array([0.03, -0.05, 0.1])
    kerr.init_uniform_field(B=tuple(B))
    h = kerr.get_contra_h()
    cen = (N - 1) / 2
    ax = np.arange(N) - cen
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    far = (np.sqrt(X * X + Y * Y + Z * Z) > 7.0)
    far[[0, -1], :, :] = far[:, [0, -1], :] = far[:, :, [0, -1]] = False
    for q in range(3):
        assert np.abs(h[q][far] - B[q]).max() < 2e-3 * np.abs(B).max(), q


def test_literal_half_steps_grow_near_the_hole_centred_stay_bounded():
    """Why the field halves are time-centred (reading A21).  In Kerr-Schild coordinates the
    covariant e of Eq. 10 depends on b through the shift terms, so taking each B half-step and the
    E step explicitly in its own start value is a forward-Euler step of a centred advection term,
    which amplifies every step.  A vacuum run around a resolved hole (32^3, m = 3, a = 0.9m, c dt =
    0.55, uniform B_z, excision at r+, outer absorbing layers so that the frozen faces add nothing)
    shows it: with the literal half-steps |d - d0| within 4m of the hole e-folds every ~13 steps
    from step ~80 (44 by step 150), while the time-centred form stays below 1."""
    N, m, steps = 32, 3.0, 150
    a = 0.9 * m
    peak = {}
    for literal in (False, True):
        rp = O.Oracle(N, N, N, m, a, 1.0, 0.55).r_plus
        o = O.Oracle(N, N, N, m, a, 1.0, 0.55, r_excise=rp, threads=0,
                     flags=O.LITERAL_HALF_STEPS if literal else 0, absorb_outer=0.2, absorb_width=5)
        o.init_uniform_field(B=(0.0, 0.0, 0.05))
        d0 = o.get_fields()[0]
        c = o.centre
        ax = [np.arange(k) - c[2 - i] for i, k in enumerate(o.shape)]
        Z, Y, X = np.meshgrid(*ax, indexing="ij")
        near = np.sqrt(X * X + Y * Y + Z * Z) < 4 * m
        hist = []
        for _ in range(steps // 25):
            o.step(25)
            hist.append(float(np.abs(o.get_fields()[0] - d0).max(axis=0)[near].max()))
        peak[literal] = hist
        o.close()
    assert max(peak[False]) < 1.0, peak[False]
    assert peak[True][-1] > 20.0, peak[True]
    # exponential, not a transient: a factor of at least 4 over each of the last two 25-step spans
    assert peak[True][-1] > 4 * peak[True][-2] > 16 * peak[True][-3], peak[True]
