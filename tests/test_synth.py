"""The seeded input generators (no GPU): positions fill the stated cells, and the momenta follow
the Maxwell-Juettner distribution they are drawn from.

* Maxwell-Juettner: f(u) ~ u^2 exp(-(gamma - 1)/theta) has <u^2> = 3 theta K3(1/theta) / K2(1/theta)
  (modified Bessel functions; scipy), checked at a thermal, a warm and a relativistic theta, with
  the directions isotropic (mean zero, equal component variances);
* uniform positions: exactly ppc particles in every cell of [1, n-3]^3, cell-major order, none
  inside r_min of the centre when asked;
* the plasma builders: species co-located, ids 0..n-1, macro charges of the species' signs.
"""
import numpy as np
import pytest

from paper_0904_0232_gb300 import synth


@pytest.mark.parametrize("theta", [0.0025, 0.05, 1.0])
def test_maxwell_juettner_second_moment(theta):
    special = pytest.importorskip("scipy.special")
    n = 400_000
    u = synth.maxwell_juettner(synth._rng(11, 3), n, theta)
    assert u.shape == (3, n)
    u2 = (u * u).sum(0)
    want = 3.0 * theta * special.kve(3, 1.0 / theta) / special.kve(2, 1.0 / theta)
    # relative standard error of the sample mean of u^2 is about sqrt(var(u^2)) / (mean sqrt(n)) < 0.3 %
    assert abs(u2.mean() / want - 1.0) < 0.01, (u2.mean(), want)
    comp_var = (u * u).mean(1)
    assert np.allclose(comp_var, want / 3.0, rtol=0.02)
    assert np.abs(u.mean(1)).max() < 5.0 * np.sqrt(want / 3.0 / n)


def test_maxwell_juettner_is_not_the_plain_gaussian():
    """At theta = 1 the relativistic tail makes <u^2> about 3 K3(1)/K2(1) ~ 7.65, far from 3."""
    u = synth.maxwell_juettner(synth._rng(2, 2), 100_000, 1.0)
    assert (u * u).sum(0).mean() > 6.5


def test_uniform_positions_fill_the_cells():
    n, ppc = 10, 3
    x = synth.uniform_positions(synth._rng(5, 0), n, n, n, ppc)
    cells = np.floor(x).astype(int)
    assert x.shape == (3, ppc * (n - 3) ** 3)
    assert cells.min() >= 1 and cells.max() <= n - 3
    idx = (cells[2] * n + cells[1]) * n + cells[0]
    assert np.all(np.diff(idx) >= 0)  # cell-major: z slowest, x fastest
    counts = np.bincount(idx, minlength=n ** 3)
    inner = counts.reshape(n, n, n)[1:n - 2, 1:n - 2, 1:n - 2]
    assert inner.min() == ppc and inner.max() == ppc and counts.sum() == inner.sum()
    r_min = 2.5
    xr = synth.uniform_positions(synth._rng(5, 0), n, n, n, ppc, r_min=r_min)
    cen = (n - 1) / 2
    assert (((xr - cen) ** 2).sum(0) >= r_min * r_min).all() and xr.shape[1] < x.shape[1]


def test_plasma_species_are_co_located():
    wl = synth.kerr_ion_electron_128(seed=3, n=12)
    e, i = wl.species
    assert np.array_equal(e.x4, i.x4) and np.all(e.x4[3] == 0.0)
    assert np.array_equal(e.ids, np.arange(e.ids.size, dtype=np.uint32))
    assert e.q_over_m == -1.0 and i.q_over_m == 1.0 / 20.0
    assert e.q_macro < 0.0 < i.q_macro and e.q_macro == -i.q_macro
    assert wl.n_particles == 2 * 8 * 9 ** 3
