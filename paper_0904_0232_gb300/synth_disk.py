"""Seeded synthetic accretion-disk plasma generated on the device (the largest workload: a 384^3
Kerr grid with ~1e9 particles, too large to draw on the host).

Like ``synth``, this module holds none of the method's arithmetic: it draws positions and
initial spatial four-velocity components; the library completes u^4 (Eq. 7) and converts the
initial field itself.

Recipe (stands in for the disk/corona set-up of Sec. 6, which has no released data):
  * Kerr a = 0.95 m, m = 8 cells at 384^3 (lengths scale with the grid edge n: m = 8 n / 384),
    centre of mass at ((n-1)/2, ...), c = 1, dt = 0.4, uniform contravariant B_z = 0.1;
  * disk: cells with |z| < 0.1 r_cyl and 6m <= r_cyl <= 150 n/384 (cell centres), relative
    density 6m / r_cyl; corona: every other cell of [1, n-3]^3 whose centre lies outside
    R = r_+ + 1, relative density 0.01;
  * electron-ion pairs (q/m = -1 and +1/20) co-located; expected pairs per cell = relative
    density x n0 / 2, n0 (particles per cell at the disk's inner edge, both species) chosen so
    that the expected total is `target`; each cell's count is the floor of its expectation
    plus one with the probability of the remainder; positions uniform inside the cell;
  * disk velocities: prograde Keplerian coordinate speed v = c sqrt(m / r_cyl) (in the sense of
    the hole's frame dragging, -phi for this metric's spin sign), u^i = gamma v^i plus an
    isotropic normal thermal spread u_th = 0.05 c per component, given as contravariant spatial
    components; corona: the normal observer's u_i = 0 plus the same thermal spread, given as
    covariant spatial components;
  * macro-particle charge chosen so that omega_p dt = wp_dt (0.025) at the inner-edge density;
  * absorbing layers (``layers``): 0.3 per step inside the horizon (r_+/2 <= r < r_+), 0.2 per
    step over the 8 cells next to the frozen faces.  With the inside of the horizon frozen, this
    spin resolved by m = 8 cells grows a field mode next to the horizon (|d| x 1e4 in 500 steps,
    the same in FP64 and at half the timestep);
  * randomness from one seeded torch generator on the device, in a fixed order of draws.
The four species are: 0 disk electrons, 1 disk ions, 2 corona electrons, 3 corona ions.
"""
from __future__ import annotations

import dataclasses
import math

GRPIC_U_COV_SPATIAL, GRPIC_U_CONTRA_SPATIAL = 1, 2


@dataclasses.dataclass
class DeviceSpecies:
    name: str
    q_over_m: float
    q_macro: float
    x4: object     # torch float64 (4, n) on the device (x^4 = 0)
    u4: object     # torch float64 (4, n): spatial components in rows 0-2, row 3 zero
    ids: object    # torch int32 (n,)
    umode: int     # how rows 0-2 of u4 are meant (GRPIC_U_COV_SPATIAL / GRPIC_U_CONTRA_SPATIAL)


@dataclasses.dataclass
class DiskCorona:
    name: str
    n: int
    m: float
    a: float
    c: float
    dt: float
    B0: float
    nsteps: int
    n0: float
    species: list
    layers: dict = dataclasses.field(default_factory=lambda: dict(absorb_inner=0.3, absorb_outer=0.2,
                                                                  absorb_width=8))

    @property
    def nx(self):
        return self.n

    ny = nz = nx

    @property
    def n_particles(self) -> int:
        return sum(int(s.ids.numel()) for s in self.species)


def _charge(dt, pairs_per_cell, qms, wp_dt):
    return (wp_dt / dt) ** 2 / (4.0 * math.pi * pairs_per_cell * sum(abs(q) for q in qms))


def kerr_disk_corona(n=384, seed=3, target=1.0e9, device="cuda", u_th=0.05, wp_dt=0.025, nsteps=500):
    import torch

    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    f64 = torch.float64
    m = 8.0 * n / 384.0
    a = 0.95 * m
    c, dt, B0 = 1.0, 0.4, 0.1
    cen = 0.5 * (n - 1)
    r_in, r_out = 6.0 * m, 150.0 * n / 384.0
    r_plus = m + math.sqrt(m * m - a * a)
    w = n - 3  # cells 1 .. n-3 per axis
    ax = torch.arange(1, n - 2, device=dev, dtype=f64) + 0.5 - cen
    # relative density per cell, z-major (cell index (k * w + j) * w + i over the interior)
    Z = ax.view(w, 1, 1)
    Y = ax.view(1, w, 1)
    X = ax.view(1, 1, w)
    rc = torch.sqrt(X * X + Y * Y)
    R = torch.sqrt(X * X + Y * Y + Z * Z)
    disk = (Z.abs() < 0.1 * rc) & (rc >= r_in) & (rc <= r_out)
    rel_disk = torch.where(disk, r_in / rc.clamp(min=1e-9), torch.zeros((), device=dev, dtype=f64))
    rel_cor = torch.where(~disk & (R > r_plus + 1.0), torch.full((), 0.01, device=dev, dtype=f64),
                          torch.zeros((), device=dev, dtype=f64))
    del rc, R, disk
    n0 = target / float((rel_disk.sum() + rel_cor.sum()).item())  # particles per cell at the inner edge
    q = _charge(dt, 0.5 * n0, (-1.0, 1.0 / 20.0), wp_dt)
    species = []
    id0 = 0
    for part, rel in (("disk", rel_disk), ("corona", rel_cor)):
        lam = (rel * (0.5 * n0)).reshape(-1)
        cnt = torch.floor(lam)
        cnt = (cnt + (torch.rand(lam.shape, generator=gen, device=dev, dtype=f64) < lam - cnt)).to(torch.int64)
        del lam
        cells = torch.repeat_interleave(torch.arange(cnt.numel(), device=dev), cnt)
        del cnt
        npairs = int(cells.numel())
        x4 = torch.zeros((4, npairs), device=dev, dtype=f64)
        x4[0] = (cells % w).to(f64) + 1.0
        x4[1] = ((cells // w) % w).to(f64) + 1.0
        x4[2] = (cells // (w * w)).to(f64) + 1.0
        del cells
        x4[:3] += torch.rand((3, npairs), generator=gen, device=dev, dtype=f64)
        ids = torch.arange(id0, id0 + npairs, device=dev, dtype=torch.int64).to(torch.int32)
        id0 += npairs
        if part == "disk":
            dx, dy = x4[0] - cen, x4[1] - cen
            rcyl = torch.sqrt(dx * dx + dy * dy)
            v = torch.sqrt(m / rcyl).clamp(max=0.5) * c
            gam = 1.0 / torch.sqrt(1.0 - (v / c) ** 2)
            base = torch.stack([gam * v * dy / rcyl, -gam * v * dx / rcyl, torch.zeros_like(v)])
            del dx, dy, rcyl, v, gam
            umode = GRPIC_U_CONTRA_SPATIAL
        else:
            base = torch.zeros((3, npairs), device=dev, dtype=f64)
            umode = GRPIC_U_COV_SPATIAL
        for qm, sname in ((-1.0, "electrons"), (1.0 / 20.0, "ions")):
            u4 = torch.zeros((4, npairs), device=dev, dtype=f64)
            u4[:3] = base + u_th * c * torch.randn((3, npairs), generator=gen, device=dev, dtype=f64)
            species.append(DeviceSpecies(f"{part} {sname}", qm, math.copysign(q, qm), x4, u4, ids, umode))
        del base
    return DiskCorona(f"kerr_disk_corona_{n}", n, m, a, c, dt, B0, nsteps, n0, species)
