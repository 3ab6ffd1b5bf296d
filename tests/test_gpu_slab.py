"""One run split into z-slabs, each slab a library context (paper_0904_0232_gb300/slab.py), all slabs
in one process on one GPU and stepped in lockstep (the messages handed over in memory, the same
messages a multi-GPU run would send between ranks).

* FP64, three slabs, five whole steps of a pair plasma around a = 0.9m whose hole lies next to the
  slab boundaries: every particle and every owned field value against the oracle on one grid, to
  FP64 rounding (1e-12);
* FP32-mixed, two slabs: against the same run on one library context, within the FP32 bounds (the
  workload drops the particles whose zig-zag split the oracle decides within 1e-4 of a face).
"""
import numpy as np
import pytest

import oracle as O
from parity_util import TOL, rel_l2, well_conditioned
from paper_0904_0232_gb300 import synth
from paper_0904_0232_gb300.grpic import (GRPIC_FIELD_B, GRPIC_FIELD_D, GRPIC_FIELD_J, GRPIC_U_FULL, GrpicError,
                                         Simulation)
from paper_0904_0232_gb300.slab import LibraryEngine, LocalTransport, SlabPlan, SlabRun, library_slab

pytestmark = pytest.mark.gpu
N, STEPS = 16, 5


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _workload():
    return synth.plasma("slab", N, 2.0, 1.8, 1.0, 0.4, 0.1, STEPS, 2, (-1.0, 1.0), 0.15, seed=31, r_min=3.0)


def _start(wl):
    """The oracle on one grid at the start (u^a completed), for the initial particles of every run."""
    ref = O.Oracle(N, N, N, wl.m, wl.a, wl.c, wl.dt, threads=0)
    ref.init_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        ref.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=sp.umode)
    return ref


def _slab_runs(wl, nslabs, prec):
    plan = SlabPlan(N, nslabs)
    start = _start(wl)
    species = [(sp.q_over_m, sp.q_macro) for sp in wl.species]
    runs = []
    for r in range(nslabs):
        lo, _ = plan.local(r)
        z0, z1 = plan.owned(r)
        sim = library_slab(plan, r, N, N, wl.m, wl.a, wl.c, wl.dt, precision=prec)
        sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
        for s, (qm, qmac) in enumerate(species):
            x4, u4, ids = start.get_particles(s)
            sel = (x4[2] >= z0) & (x4[2] < z1)
            x = x4[:, sel].copy()
            x[2] -= lo
            sim.load_particles(s, qm, qmac, x, u4[:, sel], ids[sel], umode=GRPIC_U_FULL)
        runs.append(SlabRun(plan, r, LibraryEngine(sim), species))
    return plan, runs


def _gather(runs, nspecies):
    """The owned planes of every slab stacked into the run's grid, and every particle (global z)."""
    d = np.concatenate([r.engine.get_fields()[0][:, r.z0 - r.lo:r.z1 - r.lo] for r in runs], axis=1)
    b = np.concatenate([r.engine.get_fields()[1][:, r.z0 - r.lo:r.z1 - r.lo] for r in runs], axis=1)
    J = np.concatenate([r.engine.get_fields()[2][:, r.z0 - r.lo:r.z1 - r.lo] for r in runs], axis=1)
    parts = []
    for s in range(nspecies):
        xs, us, ids = [], [], []
        for r in runs:
            x4, u4, i = r.engine.get_particles(s)
            x = x4.copy()
            x[2] += r.lo
            xs.append(x)
            us.append(u4)
            ids.append(i)
        x, u, i = np.hstack(xs), np.hstack(us), np.concatenate(ids)
        o = np.argsort(i)
        parts.append((x[:, o], u[:, o], i[o]))
    return d, b, J, parts


def test_fp64_slabs_against_the_oracle():
    wl = _workload()
    plan, runs = _slab_runs(wl, 3, "fp64")
    LocalTransport(runs).step(STEPS)
    d, b, J, parts = _gather(runs, len(wl.species))
    ref = _start(wl)
    ref.step(STEPS)
    dr, br, Jr = ref.get_fields()
    for A, B in ((d, dr), (b, br), (J, Jr)):
        assert np.abs(A - B).max() < 1e-12 * np.abs(B).max()
    crossed = 0
    for s, (x, u, i) in enumerate(parts):
        xr, ur, ir = ref.get_particles(s)
        o = np.argsort(ir)
        assert np.array_equal(i, ir[o])
        assert np.abs(x[:3] - xr[:3, o]).max() < 1e-12 * N
        assert np.abs(u - ur[:, o]).max() < 1e-12 * np.abs(ur).max()
        z0 = dict(zip(wl.species[s].ids.tolist(), wl.species[s].x4[2].tolist()))
        crossed += sum(1 for k, z in zip(i.tolist(), x[2].tolist())
                       if any((a <= z0[k] < c) != (a <= z < c) for a, c in plan.bounds))
    assert crossed > 0, "no particle changed slab: the migration went untested"


def test_fp32_mixed_slabs_against_one_context():
    wl = well_conditioned(_workload(), STEPS, threads=0)
    plan, runs = _slab_runs(wl, 2, "fp32_mixed")
    LocalTransport(runs).step(STEPS)
    d, b, J, parts = _gather(runs, len(wl.species))
    start = _start(wl)
    one = Simulation(N, N, N, wl.m, wl.a, wl.c, wl.dt, precision="fp32_mixed")
    one.set_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        x4, u4, ids = start.get_particles(s)
        one.load_particles(s, sp.q_over_m, sp.q_macro, x4, u4, ids, umode=GRPIC_U_FULL)
    one.step(STEPS)
    d1, b1, J1 = one.get_fields()
    tol = TOL["fp32_mixed"]
    assert rel_l2(J, J1) <= tol["J"] and rel_l2(b, b1) <= tol["fields"] and rel_l2(d, d1) <= max(tol["fields"], tol["J"])
    for s, (x, u, i) in enumerate(parts):
        x1, u1, i1 = one.get_particles(s)
        o = np.argsort(i1)
        assert np.array_equal(i, i1[o])
        assert np.abs(x[:3] - x1[:3, o]).max() <= tol["particles"] * N
        assert np.abs(u - u1[:, o]).max() <= tol["particles"] * max(1.0, np.abs(u1).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_planes(prec):
    """grpic_get_planes / grpic_set_planes: the planes of grpic_get_fields, written back exactly (FP32
    values round-trip), J added into; ranges outside the grid and adding into d or b are refused."""
    sim = Simulation(12, 10, 16, 2.0, 1.0, 1.0, 0.4, precision=prec)
    rng = np.random.default_rng(3)
    d0, b0, J0 = (rng.standard_normal((3, 16, 10, 12)) for _ in range(3))
    sim.set_fields(d0, b0)
    sim.set_j(J0)
    d, b, J = sim.get_fields()
    for which, F in ((GRPIC_FIELD_D, d), (GRPIC_FIELD_B, b), (GRPIC_FIELD_J, J)):
        assert np.array_equal(sim.get_planes(which, 5, 4), F[:, 5:9])
    new = rng.standard_normal((3, 3, 10, 12))
    sim.set_planes(GRPIC_FIELD_B, 0, new)
    sim.set_planes(GRPIC_FIELD_J, 13, new, add=True)
    d1, b1, J1 = sim.get_fields()
    assert np.array_equal(d1, d)
    tol = 0.0 if prec == "fp64" else 1e-7
    assert np.abs(b1[:, :3] - new).max() <= tol * np.abs(new).max() and np.array_equal(b1[:, 3:], b[:, 3:])
    assert np.allclose(J1[:, 13:], J[:, 13:] + new, rtol=1e-15, atol=0) and np.array_equal(J1[:, :13], J[:, :13])
    with pytest.raises(GrpicError):
        sim.get_planes(GRPIC_FIELD_D, 14, 3)
    with pytest.raises(GrpicError):
        sim.set_planes(GRPIC_FIELD_D, 0, new, add=True)
    sim.close()
