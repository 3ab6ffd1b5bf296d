"""One run split into z-slabs (paper_0904_0232_gb300/slab.py), on the CPU with the oracle as each
slab's engine: the split run against the same run on one grid.

* the plan: owned ranges, local planes and the minimum slab size;
* three slabs in one process (LocalTransport) and two or three gloo ranks (DistTransport,
  point-to-point messages only), each over five whole steps of a pair plasma around a = 0.9m whose hole lies next
  to the slab boundaries: every particle (matched by id) and every field value of the owned planes
  agree with the single grid to FP64 rounding.  The one difference in arithmetic is the order in
  which J at a node next to a boundary adds up (the neighbour's share is added as one sum), so the
  check is at 1e-12, not bitwise.
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
from paper_0904_0232_gb300 import synth
from paper_0904_0232_gb300.slab import DistTransport, LocalTransport, SlabPlan, SlabRun

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, STEPS = 16, 5


class OracleEngine:
    """The oracle as a slab engine (test infrastructure only)."""

    def __init__(self, ref):
        self.ref = ref
        self.plane_shape = ref.shape[1:]

    def get_planes(self, which, z0, n):
        d, b, J = self.ref.get_fields()
        return {"d": d, "b": b, "J": J}[which][:, z0:z0 + n].copy()

    def set_planes(self, which, z0, planes, add=False):
        d, b, J = self.ref.get_fields()
        n = planes.shape[1]
        if which == "J":
            if add:
                J[:, z0:z0 + n] += planes
            else:
                J[:, z0:z0 + n] = planes
            self.ref.set_j(J)
        else:
            assert not add
            (d if which == "d" else b)[:, z0:z0 + n] = planes
            self.ref.set_fields(d, b)

    def stage(self, name):
        {"b_half": self.ref.b_half, "zero_j": self.ref.zero_j, "push_deposit": self.ref.push_deposit,
         "b_half2": self.ref.b_half2, "e": self.ref.e_step, "sort": lambda: None}[name]()

    def get_fields(self):
        return self.ref.get_fields()

    def set_fields(self, d, b):
        self.ref.set_fields(d, b)

    def set_j(self, J):
        self.ref.set_j(J)

    def get_particles(self, s):
        return self.ref.get_particles(s)

    def load_particles(self, s, q_over_m, q_macro, x4, u4, ids):
        self.ref.load_particles(s, q_over_m, q_macro, x4, u4, ids, umode=0)


def _workload():
    return synth.plasma("slab", N, 2.0, 1.8, 1.0, 0.4, 0.1, STEPS, 2, (-1.0, 1.0), 0.15, seed=31, r_min=3.0)


def _whole(wl):
    ref = O.Oracle(N, N, N, wl.m, wl.a, wl.c, wl.dt, threads=1)
    ref.init_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        ref.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=sp.umode)
    return ref


def _slab(wl, plan, rank):
    """Rank `rank`'s oracle: its planes, the run's initial field there, its owned particles (u^a
    completed by a whole-grid oracle so that both runs start from the same numbers)."""
    lo, hi = plan.local(rank)
    z0, z1 = plan.owned(rank)
    ref = O.Oracle(N, N, hi - lo, wl.m, wl.a, wl.c, wl.dt, threads=1, z_origin=lo, nz_total=N)
    ref.init_uniform_field(B=(0.0, 0.0, wl.B0))
    start = _whole(wl)
    for s, sp in enumerate(wl.species):
        x4, u4, ids = start.get_particles(s)
        sel = (x4[2] >= z0) & (x4[2] < z1)
        x = x4[:, sel].copy()
        x[2] -= lo
        ref.load_particles(s, sp.q_over_m, sp.q_macro, x, u4[:, sel], ids[sel], umode=0)
    return ref


def _owned_state(run):
    d, b, J = run.engine.get_fields()
    sl = slice(run.z0 - run.lo, run.z1 - run.lo)
    parts = []
    for s in range(len(run.species)):
        x4, u4, ids = run.engine.get_particles(s)
        x = x4.copy()
        x[2] += run.lo
        parts.append((x, u4.copy(), ids.copy()))
    return d[:, sl].copy(), b[:, sl].copy(), J[:, sl].copy(), parts


def _compare(wl, states, plan):
    ref = _whole(wl)
    ref.step(STEPS)
    d, b, J = ref.get_fields()
    scale = {"d": np.abs(d).max(), "b": np.abs(b).max(), "J": np.abs(J).max()}
    for r, (ds, bs, Js, parts) in enumerate(states):
        z0, z1 = plan.owned(r)
        for name, A, B in (("d", ds, d), ("b", bs, b), ("J", Js, J)):
            err = np.abs(A - B[:, z0:z1]).max() / scale[name]
            assert err < 1e-12, (r, name, err)
    moved = 0
    for s in range(len(wl.species)):
        xr, ur, ir = ref.get_particles(s)
        x = np.hstack([st[3][s][0] for st in states])
        u = np.hstack([st[3][s][1] for st in states])
        ids = np.concatenate([st[3][s][2] for st in states])
        o, orr = np.argsort(ids), np.argsort(ir)
        assert np.array_equal(ids[o], ir[orr]), "the split run keeps the same particles"
        assert np.abs(x[:3, o] - xr[:3, orr]).max() < 1e-12 * N
        assert np.abs(u[:, o] - ur[:, orr]).max() < 1e-12 * np.abs(ur).max()
        # the plasma does cross the slab boundaries
        z_start = wl.species[s].x4[2]
        id_start = wl.species[s].ids
        zs = dict(zip(id_start.tolist(), z_start.tolist()))
        for r in range(plan.nranks):
            z0, z1 = plan.owned(r)
            pid = states[r][3][s][2]
            moved += sum(1 for i in pid.tolist() if not (z0 <= zs[i] < z1))
    assert moved > 0


def test_plan():
    p = SlabPlan(16, 2)
    assert p.owned(0) == (0, 8) and p.owned(1) == (8, 16)
    assert p.local(0) == (0, 12) and p.local(1) == (4, 16)
    assert p.neighbours(0) == [1] and p.neighbours(1) == [0]
    q = SlabPlan(16, 3)
    assert [q.owned(r) for r in range(3)] == [(0, 5), (5, 11), (11, 16)]
    assert q.local(1) == (1, 15)
    with pytest.raises(ValueError):
        SlabPlan(16, 5)  # slabs of fewer than four planes


def test_three_slabs_in_one_process():
    wl = _workload()
    plan = SlabPlan(N, 3)
    runs = [SlabRun(plan, r, OracleEngine(_slab(wl, plan, r)), [(sp.q_over_m, sp.q_macro) for sp in wl.species])
            for r in range(3)]
    LocalTransport(runs).step(STEPS)
    _compare(wl, [_owned_state(r) for r in runs], plan)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _workload()
        plan = SlabPlan(N, world)
        run = SlabRun(plan, rank, OracleEngine(_slab(wl, plan, rank)), [(sp.q_over_m, sp.q_macro) for sp in wl.species])
        DistTransport(run).step(STEPS)
        out.put((rank, _owned_state(run)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks(world):
    """One slab per process, point-to-point messages over gloo (three ranks: the middle one exchanges
    with both neighbours)."""
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _compare(_workload(), [res[r] for r in range(world)], SlabPlan(N, world))
