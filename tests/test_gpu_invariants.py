"""Invariant statistics on the device (grpic_get_invariants) against the same statistics computed
on the host from the particles read back, with the oracle's metric (Eqs. 4-6):
N = |g_mn u^m u^n + c^2| / c^2 over every live particle (Eq. 7), and for the tracked subsample
(ids divisible by 64) the changes of E = -u_4 and L = x u_y - y u_x (covariant; Eq. 3) since the
baseline.  Field-free orbits keep all three to the integrator's accuracy."""
import numpy as np
import pytest

import oracle as O
from paper_0904_0232_gb300 import synth
from paper_0904_0232_gb300.grpic import GRPIC_U_COV_SPATIAL, Simulation

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _host_invariants(sim, wl):
    out = {}
    cen = np.array([(wl.nx - 1) / 2, (wl.ny - 1) / 2, (wl.nz - 1) / 2])
    norms = []
    for s in range(len(wl.species)):
        x, u, ids = sim.get_particles(s)
        for k in range(ids.size):
            X = x[:3, k] - cen
            g = O.metric(X, wl.m, wl.a)
            uc = g @ u[:, k]
            norms.append(abs(u[:, k] @ uc + wl.c ** 2) / wl.c ** 2)
            if ids[k] % 64 == 0:
                out[(s, int(ids[k]))] = (-uc[3], X[0] * uc[1] - X[1] * uc[0])
    return np.array(norms), out


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_device_statistics_match_host(prec):
    wl = synth.plasma("inv", 24, 2.0, 1.6, 1.0, 0.4, 0.08, 3, 2, (-1.0, 0.05), 0.1, seed=21, r_min=4.4)
    sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision=prec)
    sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        sim.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=GRPIC_U_COV_SPATIAL)
    base = sim.invariants(baseline=True)
    n0, inv0 = _host_invariants(sim, wl)
    assert base["n"] == n0.size
    assert base["norm_max"] == pytest.approx(n0.max(), rel=1e-6, abs=1e-15)
    sim.step(4)
    now = sim.invariants()
    n1, inv1 = _host_invariants(sim, wl)
    common = sorted(set(inv0) & set(inv1))
    assert now["tracked"] == len(common) > 50
    dE = np.array([abs(inv1[k][0] - inv0[k][0]) for k in common]) / wl.c
    dL = np.array([abs(inv1[k][1] - inv0[k][1]) for k in common]) / wl.c
    assert now["n"] == n1.size
    assert now["norm_max"] == pytest.approx(n1.max(), rel=1e-6, abs=1e-15)
    assert now["norm_mean"] == pytest.approx(n1.mean(), rel=1e-6, abs=1e-15)
    assert now["energy_max"] == pytest.approx(dE.max(), rel=1e-9, abs=1e-14)
    assert now["energy_mean"] == pytest.approx(dE.mean(), rel=1e-9, abs=1e-14)
    assert now["angmom_max"] == pytest.approx(dL.max(), rel=1e-9, abs=1e-13)
    assert now["angmom_mean"] == pytest.approx(dL.mean(), rel=1e-9, abs=1e-13)
    # the field and the plasma do work on the particles: E changes well above rounding
    assert now["energy_max"] > 1e-4


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-5), ("fp32_mixed", 2e-5)])
def test_field_free_orbits_keep_their_invariants(prec, bound):
    """Neutral test particles (no charge, no field): E, L and the norm change only by the
    integrator's error -- RK4 keeps none of them exactly, each drifts at O(h^4) per step (the
    oracle's geodesic pin), largest for the orbits that start nearest the hole (r = 6m here) --
    and by rounding, over 40 steps at dt = 0.4."""
    wl = synth.plasma("geo", 32, 1.0, 0.7, 1.0, 0.4, 0.0, 3, 1, (1.0,), 0.1, seed=22, r_min=6.0)
    sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision=prec)
    sp = wl.species[0]
    sim.load_particles(0, 0.0, 0.0, sp.x4, sp.usp * 0.3, sp.ids, umode=GRPIC_U_COV_SPATIAL)
    sim.invariants(baseline=True)
    sim.step(40)
    now = sim.invariants()
    assert now["tracked"] > 100
    assert now["energy_max"] <= bound and now["angmom_max"] <= bound * 20
    assert now["norm_max"] <= 1e-4
