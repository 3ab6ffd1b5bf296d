"""The seeded stand-in for the application set-up of Sec. 6 (synth.kerr_jet_disk) has the
parameters and structure that section states: 0.8 million disk particles at 100 times the
corona's density, the disk at R > 3 r_S with |cos theta| < 1/8, Keplerian speeds turning with
the hole's frame dragging (its sense taken from the oracle's metric), co-located pairs, and the
stated omega_p dt at the disk's density."""
import numpy as np

import oracle as O
from paper_0904_0232_gb300 import synth


def _wl():
    return synth.kerr_jet_disk(seed=4)


def test_parameters_and_counts():
    wl = _wl()
    assert (wl.nx, wl.ny, wl.nz) == (64, 64, 128)
    assert (wl.c, wl.dt, wl.B0) == (0.05, 1.0, 30.0)
    assert abs(wl.a - 0.95 * wl.m) < 1e-15
    disk_e, disk_p, cor_e, cor_p = wl.species
    assert abs(disk_e.ids.size + disk_p.ids.size - 800_000) < 0.005 * 800_000
    for e, p in ((disk_e, disk_p), (cor_e, cor_p)):
        assert np.array_equal(e.x4, p.x4) and np.array_equal(e.ids, p.ids)
        assert e.q_over_m == -1e-3 and p.q_over_m == 1e-3 and e.q_macro == -p.q_macro
    ids = np.concatenate([disk_e.ids, cor_e.ids])
    assert np.unique(ids).size == ids.size
    # omega_p dt at the disk density: sum over species of 4 pi n |q| |q/m| = (wp_dt / dt)^2
    cen = np.array([(wl.nx - 1) / 2, (wl.ny - 1) / 2, (wl.nz - 1) / 2]).reshape(3, 1)
    cells = np.floor(disk_e.x4[:3]).astype(int)
    n_cells = np.unique(cells[0] + 64 * (cells[1] + 64 * cells[2])).size
    n_disk = (disk_e.ids.size + disk_p.ids.size) / n_cells
    wp2 = 4 * np.pi * n_disk * abs(disk_e.q_macro) * 1e-3
    assert abs(np.sqrt(wp2) * wl.dt - 0.025) < 0.025 * 0.01
    # geometry: disk cells at R > 3 r_S = 6 m, |cos theta| < 1/8; corona outside R = r_+ + 1
    Xc = cells + 0.5 - cen
    R = np.sqrt((Xc ** 2).sum(0))
    assert (R > 6 * wl.m).all() and (np.abs(Xc[2]) < R / 8).all()
    cc = np.floor(cor_e.x4[:3]).astype(int) + 0.5 - cen
    Rc = np.sqrt((cc ** 2).sum(0))
    rp = wl.m + np.sqrt(wl.m ** 2 - wl.a ** 2)
    assert (Rc > rp + 1).all()
    inside = (Rc > 6 * wl.m) & (np.abs(cc[2]) < Rc / 8)
    assert not inside.any()
    # corona density 1 % of the disk's (counts over the corona's cells)
    n_cor_cells = 0
    X = np.stack(np.meshgrid(np.arange(1, 62), np.arange(1, 62), np.arange(1, 126), indexing="ij")).reshape(3, -1)
    Xm = X + 0.5 - cen
    RR = np.sqrt((Xm ** 2).sum(0))
    n_cor_cells = (~((RR > 6 * wl.m) & (np.abs(Xm[2]) < RR / 8)) & (RR > rp + 1)).sum()
    ratio = (disk_e.ids.size / n_cells) / (cor_e.ids.size / n_cor_cells)
    assert abs(ratio - 100.0) < 3.0


def test_disk_is_keplerian_and_prograde():
    wl = _wl()
    sp = wl.species[0]
    assert sp.umode == synth.GRPIC_U_CONTRA_SPATIAL and wl.species[2].umode == synth.GRPIC_U_COV_SPATIAL
    cen = np.array([(wl.nx - 1) / 2, (wl.ny - 1) / 2, (wl.nz - 1) / 2]).reshape(3, 1)
    X = sp.x4[:3] - cen
    R = np.sqrt((X ** 2).sum(0))
    rc = np.sqrt(X[0] ** 2 + X[1] ** 2)
    u_phi = (-X[1] * sp.usp[0] + X[0] * sp.usp[1]) / rc  # contravariant, along +phi
    v = wl.c * np.sqrt(wl.m / R)
    expect = -v / np.sqrt(1 - (v / wl.c) ** 2)  # turning along -phi
    # the thermal spread (0.05 c per component) averages out over a radial bin
    for lo in (14.0, 20.0, 26.0):
        sel = (R > lo) & (R < lo + 2)
        assert abs((u_phi[sel] - expect[sel]).mean()) < 0.002 * wl.c
    # frame dragging turns the same way: omega = -g_4phi / g_phiphi in the equatorial plane
    for r in (14.0, 24.0):
        for ang in (0.3, 2.0, 4.0):
            P = np.array([r * np.cos(ang), r * np.sin(ang), 0.0])
            g = O.metric(P, wl.m, wl.a)
            ephi = np.array([-P[1], P[0], 0.0])
            g4phi = ephi @ g[:3, 3]
            gphiphi = ephi @ g[:3, :3] @ ephi
            assert -g4phi / gphiphi < 0.0
