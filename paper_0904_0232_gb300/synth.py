"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the method's arithmetic (no metric, no field conversion): it draws
positions and covariant spatial four-velocity components; each implementation completes u^4
and converts the initial field itself.  Both the CUDA path and the oracle take these inputs.

Recipe (stands in for the disk/corona set-ups of Sec. 6, which have no released data):
  * positions uniform inside each cell of [1, n-3]^3 (so inside [1, n-2]), ``ppc`` per cell
    and species, optionally skipping particles within Euclidean distance ``r_min`` of the
    centre; pair plasmas are co-located (net charge density zero at start);
  * covariant spatial momenta u_i / c isotropic with |u| drawn from the Maxwell-Juettner
    distribution f(u) ~ u^2 exp(-(sqrt(1+u^2) - 1)/theta), theta = (u_th / c)^2, by inverse
    transform of a tabulated CDF;
  * macro-particle charge chosen so that the plasma frequency at the loaded density gives a
    stated omega_p dt (Sec. 5 requires omega_p dt < 2); the Kerr electron-ion workload uses
    0.025, low enough that the charge-separation field near the hole stays bounded for 500
    steps at dt = 0.4;
  * the RNG is numpy's counter-based Philox keyed by (seed, species).
"""
from __future__ import annotations

import dataclasses

import numpy as np


GRPIC_U_COV_SPATIAL, GRPIC_U_CONTRA_SPATIAL = 1, 2


@dataclasses.dataclass
class SpeciesInput:
    q_over_m: float
    q_macro: float
    x4: np.ndarray   # (4, n) grid coordinates, x^4 = 0
    usp: np.ndarray  # (3, n) spatial four-velocity components, meant as umode says
    ids: np.ndarray  # (n,) uint32
    umode: int = GRPIC_U_COV_SPATIAL  # covariant u_i, or contravariant u^i (GRPIC_U_CONTRA_SPATIAL)


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    m: float
    a: float
    c: float
    dt: float
    B0: float
    nsteps: int
    species: list

    @property
    def n_particles(self) -> int:
        return sum(s.ids.size for s in self.species)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def maxwell_juettner(rng: np.random.Generator, n: int, theta: float) -> np.ndarray:
    """(3, n) isotropic momenta per unit mass (units of c) with |u| ~ u^2 exp(-(gamma-1)/theta)."""
    if n == 0:
        return np.zeros((3, 0))
    umax = np.sqrt((1.0 + 40.0 * theta) ** 2 - 1.0)
    u = np.linspace(0.0, umax, 20001)
    pdf = u * u * np.exp(-(np.sqrt(1.0 + u * u) - 1.0) / theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(u))])
    cdf /= cdf[-1]
    mag = np.interp(rng.random(n), cdf, u)
    d = rng.standard_normal((3, n))
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    return d * mag


def uniform_positions(rng, nx, ny, nz, ppc, r_min=0.0, cells=None):
    """(3, n) positions, ppc per cell in cells [1, n-3]^3 (or the given (i, j, k) cell list)."""
    if cells is None:
        ci, cj, ck = np.meshgrid(np.arange(1, nx - 2), np.arange(1, ny - 2), np.arange(1, nz - 2), indexing="ij")
        cells = np.stack([ci.ravel(), cj.ravel(), ck.ravel()])
        order = np.lexsort((cells[0], cells[1], cells[2]))
        cells = cells[:, order]
    base = np.repeat(cells, ppc, axis=1).astype(np.float64)
    x = base + rng.random(base.shape)
    if r_min > 0.0:
        cen = np.array([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2]).reshape(3, 1)
        keep = ((x - cen) ** 2).sum(0) >= r_min * r_min
        x = x[:, keep]
    return x


def charge_for(dt, ppc, q_over_m_list, wp_dt=0.25):
    """|q_macro| with sum_s 4 pi ppc |q_macro| |q/m|_s = (wp_dt / dt)^2."""
    return (wp_dt / dt) ** 2 / (4.0 * np.pi * ppc * sum(abs(q) for q in q_over_m_list))


def plasma(name, n, m, a, c, dt, B0, nsteps, ppc, qms, u_th, seed, r_min=0.0, max_particles=None, cells=None,
           wp_dt=0.25):
    rng = _rng(seed, 0)
    x = uniform_positions(rng, n, n, n, ppc, r_min=r_min, cells=cells)
    if max_particles is not None and x.shape[1] > max_particles:
        x = x[:, :max_particles]
    npart = x.shape[1]
    x4 = np.vstack([x, np.zeros((1, npart))])
    q = charge_for(dt, ppc, qms, wp_dt)
    theta = (u_th / c) ** 2
    species = []
    for s, qm in enumerate(qms):
        usp = maxwell_juettner(_rng(seed, 1 + s), npart, theta) * c
        species.append(SpeciesInput(q_over_m=qm, q_macro=float(np.sign(qm) * q), x4=x4.copy(), usp=usp,
                                    ids=np.arange(npart, dtype=np.uint32)))
    return Workload(name, n, n, n, m, a, c, dt, B0, nsteps, species)


def schwarzschild_pairs_32(seed=1, max_particles=None):
    """a = 0, m = 2 cells, 32^3, e-/e+ pairs (q/m = -1, +1), 2 per cell per species outside
    R = 3m, Maxwell-Juettner u_th = 0.1 c, uniform B_z = 0.05, dt = 0.4, 20 steps."""
    return plasma("schwarzschild_pairs_32", 32, 2.0, 0.0, 1.0, 0.4, 0.05, 20, 2, (-1.0, 1.0), 0.1, seed,
                  r_min=6.0, max_particles=max_particles)


def kerr_ion_electron_128(seed=2, max_particles=None, n=128, cells=None, wp_dt=0.025):
    """a = 0.9 m, m = 4 cells, 128^3, electrons (q/m = -1) and ions (q/m = +1/20), 8 per cell
    per species, u_th = 0.05 c, uniform B_z = 0.1, dt = 0.4, 200 steps, omega_p dt = wp_dt."""
    return plasma(f"kerr_ion_electron_{n}", n, 4.0, 3.6, 1.0, 0.4, 0.1, 200, 8, (-1.0, 1.0 / 20.0), 0.05, seed,
                  max_particles=max_particles, cells=cells, wp_dt=wp_dt)


def kerr_jet_disk(seed=4, m=2.0, n_disk=800_000, u_th=0.05, wp_dt=0.025, nsteps=500):
    """The application set-up of Sec. 6, with its parameters where it gives them: a 64 x 64 x 128
    grid, c = 0.05 with dt = 1 (the Stoney standard dx = dt = 1), spin a = 0.95 m co-rotating with
    the disk, a Keplerian disk at R > r_d = 3 r_S and |cos theta| < 1/8 holding 100 times the
    corona's particle density and 0.8 million particles, a free-falling corona, contravariant
    B_z = 30, electron-positron pairs with |q/m| = 1e-3, 500 steps.

    Readings where the paper leaves a choice: the Stoney unit charge is not given, so the mass in
    cells is a parameter (m = 2: r_S = 2 m = 4 cells, r_d = 12 cells); the disk geometry and the
    Keplerian speed v = c sqrt(r_S / 2R) = c sqrt(m / R) use the coordinate radius R = |x - X_c|
    (R and the quartic's r differ by under 1.5 % at r_d); the disk turns in the sense of the
    hole's frame dragging (-phi for this metric's spin sign), u^i = gamma v^i, given as
    contravariant spatial components; corona particles start at u_i = 0 (the observer at rest in
    the slicing falls freely) in cells whose centre lies outside R = r_+ + 1; both take an
    isotropic normal thermal spread of u_th c per component (the paper gives none); counts per
    cell are the floor of the expectation plus one with the probability of the remainder, pairs
    co-located, positions uniform in the cell, cells [1, n-3] per axis; the macro-particle charge
    gives omega_p dt = wp_dt at the disk's density.  Species: 0 disk electrons, 1 disk positrons,
    2 corona electrons, 3 corona positrons."""
    nx, ny, nz = 64, 64, 128
    c, dt, B0, qm = 0.05, 1.0, 30.0, 1e-3
    a = 0.95 * m
    r_plus = m + np.sqrt(m * m - a * a)
    cen = np.array([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2])
    ci, cj, ck = np.meshgrid(np.arange(1, nx - 2), np.arange(1, ny - 2), np.arange(1, nz - 2), indexing="ij")
    cells = np.stack([ci.ravel(), cj.ravel(), ck.ravel()])
    cells = cells[:, np.lexsort((cells[0], cells[1], cells[2]))]
    X = cells + 0.5 - cen.reshape(3, 1)
    R = np.sqrt((X ** 2).sum(0))
    disk = (R > 6.0 * m) & (np.abs(X[2]) < R / 8.0)
    corona = ~disk & (R > r_plus + 1.0)
    pairs_disk = 0.5 * n_disk / disk.sum()
    rng = _rng(seed, 0)
    species = []
    q = charge_for(dt, pairs_disk, (qm, qm), wp_dt)
    id0 = 0
    for part, sel, dens in (("disk", disk, pairs_disk), ("corona", corona, 0.01 * pairs_disk)):
        cc = cells[:, sel]
        lam = np.full(cc.shape[1], dens)
        cnt = np.floor(lam).astype(np.int64)
        cnt += rng.random(cnt.size) < lam - cnt
        x = np.repeat(cc, cnt, axis=1).astype(np.float64)
        x += rng.random(x.shape)
        npairs = x.shape[1]
        x4 = np.vstack([x, np.zeros((1, npairs))])
        ids = np.arange(id0, id0 + npairs, dtype=np.uint32)
        id0 += npairs
        if part == "disk":
            d = x[:2] - cen[:2].reshape(2, 1)
            Rp = np.sqrt(((x - cen.reshape(3, 1)) ** 2).sum(0))
            rc = np.sqrt((d ** 2).sum(0))
            v = c * np.sqrt(m / Rp)
            gam = 1.0 / np.sqrt(1.0 - (v / c) ** 2)
            base = np.vstack([gam * v * d[1] / rc, -gam * v * d[0] / rc, np.zeros(npairs)])
            umode = GRPIC_U_CONTRA_SPATIAL
        else:
            base = np.zeros((3, npairs))
            umode = GRPIC_U_COV_SPATIAL
        for sign in (-1.0, 1.0):
            usp = base + u_th * c * rng.standard_normal((3, npairs))
            species.append(SpeciesInput(q_over_m=sign * qm, q_macro=sign * q, x4=x4.copy(), usp=usp, ids=ids.copy(),
                                        umode=umode))
    return Workload("kerr_jet_disk_64x64x128", nx, ny, nz, m, a, c, dt, B0, nsteps, species)


def subsample(wl, n_per_species):
    """The same workload keeping n evenly strided particles per species (a bounded sample that
    still spans the whole grid)."""
    species = []
    for sp in wl.species:
        k = max(1, sp.ids.size // max(1, n_per_species))
        sel = np.arange(0, sp.ids.size, k)[:n_per_species]
        species.append(SpeciesInput(sp.q_over_m, sp.q_macro, sp.x4[:, sel].copy(), sp.usp[:, sel].copy(),
                                    sp.ids[sel].copy(), sp.umode))
    return Workload(wl.name + f"_sample{n_per_species}", wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, wl.B0,
                    wl.nsteps, species)


def random_fields(shape, seed, scale=0.05):
    """Smooth-ish random prognostic fields (d, b), each (3, nz, ny, nx)."""
    rng = _rng(seed, 99)
    d = rng.standard_normal((3,) + tuple(shape)) * scale
    b = rng.standard_normal((3,) + tuple(shape)) * scale
    return d, b


@dataclasses.dataclass
class InstanceSpec:
    grid: int
    ppc: int
    m: float
    a: float


def batch_specs(n=64, seed=7, grids=(32, 48, 64, 96), ppc_range=(1, 32), m_range=(1.0, 4.0), spin_max=0.99):
    """Parameters of n independent instances: grid drawn from `grids`, particles per cell per
    species uniform in ppc_range, m uniform in m_range (cells), a uniform in [0, spin_max] m."""
    rng = _rng(seed, 7)
    out = []
    for _ in range(n):
        g = int(grids[rng.integers(0, len(grids))])
        ppc = int(rng.integers(ppc_range[0], ppc_range[1] + 1))
        m = float(rng.uniform(*m_range))
        a = float(rng.uniform(0.0, spin_max)) * m
        out.append(InstanceSpec(g, ppc, m, a))
    return out


def cell_major_pairs(n, ppc_max, u_th, c, seed):
    """Pair-plasma draws for a grid of n^3 nodes with ppc_max particles in every cell of
    [1, n-3]^3, laid out (3, ncell, ppc_max): positions (shared by both species, co-located
    pairs) and covariant spatial momenta per species.  Taking [:, :, :ppc] gives ppc per cell."""
    rng = _rng(seed, 1000 + n)
    x = uniform_positions(rng, n, n, n, ppc_max)
    ncell = x.shape[1] // ppc_max
    theta = (u_th / c) ** 2
    u0 = maxwell_juettner(_rng(seed, 2000 + n), x.shape[1], theta) * c
    u1 = maxwell_juettner(_rng(seed, 3000 + n), x.shape[1], theta) * c
    shape = (3, ncell, ppc_max)
    return x.reshape(shape), u0.reshape(shape), u1.reshape(shape)
