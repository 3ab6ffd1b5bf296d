"""Pins of the oracle's slab option (reading A24: a grid that is planes z_origin .. z_origin + nz - 1 of
a larger run keeps the run's centre, so that a run split into slabs sees one metric).

Checked against the whole grid: one B half-step, one E step and one push + deposit of a slab reproduce
the whole grid's result wherever the stencil of a point lies inside the slab; a slab placed with a
wrong origin (the centre of its own planes) does not.  Invalid placements are refused.
"""
import numpy as np
import pytest

import oracle as O

N, M, A = 16, 2.0, 1.8
Z0, NZ = 5, 8  # the slab: global planes 5 .. 12 (off the centre)


def _fields(seed=3):
    rng = np.random.default_rng(seed)
    d = 0.05 * rng.standard_normal((3, N, N, N))
    b = 0.1 + 0.05 * rng.standard_normal((3, N, N, N))
    return d, b


def _pair(d, b, z_origin=Z0, nz_total=N):
    whole = O.Oracle(N, N, N, M, A, 1.0, 0.4, threads=2, flags=O.NO_GAMMA_TERMS)
    whole.set_fields(d, b)
    part = O.Oracle(N, N, NZ, M, A, 1.0, 0.4, threads=2, flags=O.NO_GAMMA_TERMS, z_origin=z_origin,
                    nz_total=nz_total)
    part.set_fields(d[:, Z0:Z0 + NZ], b[:, Z0:Z0 + NZ])
    return whole, part


def test_centre_of_a_slab():
    whole, part = _pair(*_fields())
    assert np.array_equal(part.centre + np.array([0.0, 0.0, Z0]), whole.centre)


@pytest.mark.parametrize("stage", ["b_half", "e_step"])
def test_field_stage_matches_whole_grid(stage):
    """B half-step: b(p) reads planes p-1 .. p+2.  E step: d(p) reads the predicted d* on planes
    p-1 .. p+1, which a grid predicts only on its advanced planes (not its two edge planes).  On the
    planes whose stencil the slab holds, its result is the whole grid's, bit for bit (the coordinates
    of lattice points are exact in both)."""
    d, b = _fields()
    whole, part = _pair(d, b)
    getattr(whole, stage)()
    getattr(part, stage)()
    dw, bw, _ = whole.get_fields()
    dp, bp, _ = part.get_fields()
    lo, hi = (Z0 + 1, Z0 + NZ - 3) if stage == "b_half" else (Z0 + 3, Z0 + NZ - 4)
    lo, hi = max(lo, Z0 + 2), min(hi, Z0 + NZ - 3)  # and advanced in the slab (not its two edge planes)
    F_w, F_p = (bw, bp) if stage == "b_half" else (dw, dp)
    assert np.array_equal(F_p[:, lo - Z0:hi - Z0 + 1], F_w[:, lo:hi + 1])
    # the stage changed those planes (the check is not vacuous)
    F0 = b if stage == "b_half" else d
    assert np.abs(F_w[:, lo:hi + 1] - F0[:, lo:hi + 1]).max() > 1e-6
    # a slab that takes the centre of its own planes computes a different metric there
    wrong = O.Oracle(N, N, NZ, M, A, 1.0, 0.4, threads=2, flags=O.NO_GAMMA_TERMS)
    wrong.set_fields(d[:, Z0:Z0 + NZ], b[:, Z0:Z0 + NZ])
    getattr(wrong, stage)()
    dx, bx, _ = wrong.get_fields()
    F_x = bx if stage == "b_half" else dx
    assert not np.allclose(F_x[:, lo - Z0:hi - Z0 + 1], F_w[:, lo:hi + 1], rtol=0, atol=1e-9)


def test_push_deposit_matches_whole_grid():
    """Particles in the middle planes of the slab: the same moves (positions shifted by the origin) and
    the same J on every node, to rounding (the particle's offset from the centre is formed from
    differently shifted coordinates)."""
    d, b = _fields(5)
    whole, part = _pair(d, b)
    rng = np.random.default_rng(7)
    n = 1200
    x = np.vstack([rng.uniform(3.0, 12.0, n), rng.uniform(3.0, 12.0, n), rng.uniform(Z0 + 2.2, Z0 + NZ - 3.2, n),
                   np.zeros(n)])
    usp = 0.2 * rng.standard_normal((3, n))
    ids = np.arange(n, dtype=np.uint32)
    # keep the particles well outside the horizon
    R = np.linalg.norm(x[:3] - whole.centre[:, None], axis=0)
    keep = R > 1.5 * whole.r_plus
    x, usp, ids = x[:, keep], usp[:, keep], ids[keep]
    xs = x.copy()
    xs[2] -= Z0
    whole.load_particles(0, -1.0, 1e-3, x, usp, ids, umode=1)
    part.load_particles(0, -1.0, 1e-3, xs, usp, ids, umode=1)
    whole.zero_j()
    part.zero_j()
    whole.push_deposit()
    part.push_deposit()
    xw, uw, iw = whole.get_particles(0)
    xp, up, ip = part.get_particles(0)
    assert np.array_equal(iw, ip) and iw.size > 300
    xp[2] += Z0
    assert np.abs(xp[:3] - xw[:3]).max() < 1e-12
    assert np.abs(up - uw).max() < 1e-12 * np.abs(uw).max()
    Jw = whole.get_fields()[2]
    Jp = part.get_fields()[2]
    assert np.abs(Jw[:, :Z0]).max() == 0.0 and np.abs(Jw[:, Z0 + NZ:]).max() == 0.0
    assert np.abs(Jp - Jw[:, Z0:Z0 + NZ]).max() < 1e-13 * np.abs(Jw).max()
    assert np.abs(Jw).max() > 0


def test_invalid_slabs_are_refused():
    with pytest.raises(ValueError):
        O.Oracle(N, N, NZ, M, A, 1.0, 0.4, z_origin=10, nz_total=N)  # runs past the last plane
    with pytest.raises(ValueError):
        O.Oracle(N, N, NZ, M, A, 1.0, 0.4, z_origin=-1, nz_total=N)
    with pytest.raises(ValueError):
        O.Oracle(N, N, NZ, M, A, 1.0, 0.4, z_origin=Z0, nz_total=N, absorb_outer=0.2)  # faces not its own
    O.Oracle(N, N, NZ, M, A, 1.0, 0.4, z_origin=Z0, nz_total=N, absorb_inner=0.3)  # the inner layer is fine
