"""One run split into z-slabs, one context per rank: halo exchange of the fields, a ghost sum of J and
particle migration, all as point-to-point messages between neighbouring slabs (no collective).

A run of nz planes is split into contiguous owned ranges [z0, z1) of at least GHOST planes each.  A
rank's context holds its owned planes plus GHOST planes of each neighbour (none past the run's first
and last plane), created with ``z_origin`` / ``nz_total`` so that its metric is the run's (the hole at
the run's centre).  Its two edge planes next to a neighbour are held by the context like faces; the
exchange keeps every plane a neighbour owns up to date instead.  One timestep (the cycle of Sec. 2.2,
Fig. 1, on every slab):

1. first B half-step (Eq. 10), then the neighbours' b in the ghost planes;
2. J = 0, push + deposit (Secs. 3.3 and 4); each slab sends the J its particles left in a neighbour's
   planes to that neighbour, which adds it to its own;
3. the owned planes' completed J next to a neighbour refresh that neighbour's ghost J (the E step's
   predictor reads J there);
4. second B half-step, then the ghost b;
5. E step (Eq. 12), then the ghost d;
6. the sort; particles that left the owned planes move to the neighbour that owns their new plane.

Why GHOST = 4: a plane's B update reads b and d of the planes p-1 .. p+2, the E step reads the
predicted d* of the planes p-1 .. p+1, which a context computes only off its two edge planes, and a
particle moves less than a cell per step (the step limit), so its push and deposit reach at most
two planes past the plane it starts in.  With the ghost planes refreshed after every field stage,
every owned plane then sees exactly what it would see in the whole run.

The engine of a rank is any object with ``stage(name)`` for the stage names below,
``get_planes(which, z0, n)`` -> a (3, n, ny, nx) float64 array of planes z0 .. z0 + n - 1 (local) of
field which in "d", "b", "J", ``set_planes(which, z0, planes, add=False)`` (add: J only),
``get_particles(s)`` -> (x4, u4, ids) with x4[2] in local planes and x^4 the particle's own clock, and
``load_particles(s, q_over_m, q_macro, x4, u4, ids)`` taking u^a as given.  ``LibraryEngine`` wraps a
library context (one GPU each; the planes move through grpic_get_planes / grpic_set_planes).  Messages
are float64 vectors; ``DistTransport`` sends them with torch.distributed point-to-point calls (gloo or
NCCL), ``LocalTransport`` hands them over within one process (all slabs in one process, e.g. one GPU
holding several contexts).  Only the GHOST planes next to a neighbour cross, through host memory.
"""
from __future__ import annotations

import numpy as np

GHOST = 4
STAGES = ("b_half", "zero_j", "push_deposit", "b_half2", "e", "sort")


class SlabPlan:
    """Owned plane ranges of `nranks` slabs of an nz-plane run, and each slab's local planes."""

    def __init__(self, nz: int, nranks: int, ghost: int = GHOST):
        if nranks < 1:
            raise ValueError("at least one slab")
        self.nz, self.nranks, self.ghost = int(nz), int(nranks), int(ghost)
        cuts = [round(r * self.nz / self.nranks) for r in range(self.nranks + 1)]
        self.bounds = [(cuts[r], cuts[r + 1]) for r in range(self.nranks)]
        for z0, z1 in self.bounds:
            if z1 - z0 < self.ghost:
                raise ValueError(f"each slab needs at least {self.ghost} planes: {nz} planes in {nranks} slabs")

    def owned(self, r: int):
        return self.bounds[r]

    def local(self, r: int):
        """Global planes [lo, hi) held by rank r's context."""
        z0, z1 = self.bounds[r]
        lo = z0 - self.ghost if r > 0 else 0
        hi = z1 + self.ghost if r < self.nranks - 1 else self.nz
        return lo, hi

    def neighbours(self, r: int):
        return [q for q in (r - 1, r + 1) if 0 <= q < self.nranks]


class SlabRun:
    """Rank r's part of a run: its engine and the messages of each phase of a step."""

    PHASES = ("b_half", "j_sum", "j_halo", "b_half2", "e", "migrate")

    def __init__(self, plan: SlabPlan, rank: int, engine, species, plane_shape=None):
        """species: list of (q_over_m, q_macro) per species index; plane_shape: (ny, nx) of the run."""
        self.plan, self.rank, self.engine = plan, rank, engine
        self.species = list(species)
        self.plane_shape = tuple(plane_shape) if plane_shape is not None else getattr(engine, "plane_shape", None)
        self.lo, self.hi = plan.local(rank)
        self.z0, self.z1 = plan.owned(rank)

    # global plane ranges a message covers, as local slices
    def _sl(self, g0, g1):
        return slice(g0 - self.lo, g1 - self.lo)

    def _ghost_of(self, peer):
        """Planes of peer that this rank holds as ghost planes."""
        return (self.z0 - self.plan.ghost, self.z0) if peer < self.rank else (self.z1, self.z1 + self.plan.ghost)

    def _edge_for(self, peer):
        """Own planes that peer holds as ghost planes."""
        return (self.z0, self.z0 + self.plan.ghost) if peer < self.rank else (self.z1 - self.plan.ghost, self.z1)

    def compute(self, phase):
        e = self.engine
        if phase == "b_half":
            e.stage("b_half")
        elif phase == "j_sum":
            e.stage("zero_j")
            e.stage("push_deposit")
        elif phase == "b_half2":
            e.stage("b_half2")
        elif phase == "e":
            e.stage("e")
        elif phase == "migrate":
            e.stage("sort")

    def outgoing(self, phase):
        """{peer: float64 vector} to send after `phase`'s compute."""
        out = {}
        peers = self.plan.neighbours(self.rank)
        e = self.engine
        if phase in ("b_half", "b_half2", "e"):
            which = "d" if phase == "e" else "b"
            for q in peers:
                g0, g1 = self._edge_for(q)
                out[q] = e.get_planes(which, g0 - self.lo, g1 - g0).ravel()
        elif phase in ("j_sum", "j_halo"):
            for q in peers:
                g0, g1 = self._ghost_of(q) if phase == "j_sum" else self._edge_for(q)
                out[q] = e.get_planes("J", g0 - self.lo, g1 - g0).ravel()
        elif phase == "migrate":
            self._moving = {}
            keep = []
            for s in range(len(self.species)):
                x4, u4, ids = e.get_particles(s)
                zg = x4[2] + self.lo
                below, above = zg < self.z0, zg >= self.z1
                stay = ~(below | above)
                keep.append((x4[:, stay], u4[:, stay], ids[stay]))
                for q, sel in ((self.rank - 1, below), (self.rank + 1, above)):
                    if sel.any() and q not in peers:
                        raise RuntimeError("a particle left the run's planes without being removed")
                    if q in peers:
                        x = x4[:, sel].copy()
                        x[2] += self.lo  # global planes on the wire
                        rec = np.vstack([np.full((1, x.shape[1]), float(s)), x, u4[:, sel],
                                         ids[sel].astype(np.float64)[None, :]])
                        self._moving.setdefault(q, []).append(rec)
            self._keep = keep
            for q in peers:
                recs = self._moving.get(q, [])
                out[q] = (np.hstack(recs) if recs else np.zeros((10, 0))).ravel(order="F")
        return out

    def incoming(self, phase, msgs):
        """Apply the neighbours' messages of `phase`."""
        e = self.engine
        if phase in ("b_half", "b_half2", "e", "j_sum", "j_halo"):
            which = {"b_half": "b", "b_half2": "b", "e": "d"}.get(phase, "J")
            for q, v in msgs.items():
                # ghost sums land on the own planes next to the sender; the rest on the ghost planes
                g0, g1 = self._edge_for(q) if phase == "j_sum" else self._ghost_of(q)
                planes = v.reshape((3, g1 - g0) + self._plane_shape(v, g1 - g0))
                e.set_planes(which, g0 - self.lo, planes, add=phase == "j_sum")
        elif phase == "migrate":
            got = [v.reshape((10, -1), order="F") for v in msgs.values()]
            for s, (qm, qmac) in enumerate(self.species):
                x4, u4, ids = self._keep[s]
                parts_x, parts_u, parts_i = [x4], [u4], [ids.astype(np.uint32)]
                for rec in got:
                    sel = rec[0] == float(s)
                    x = rec[1:5, sel].copy()
                    x[2] -= self.lo
                    parts_x.append(x)
                    parts_u.append(rec[5:9, sel])
                    parts_i.append(rec[9, sel].astype(np.uint32))
                e.load_particles(s, qm, qmac, np.hstack(parts_x), np.hstack(parts_u), np.concatenate(parts_i))
            self._keep = None

    def _plane_shape(self, v, nplanes):
        """(ny, nx) of a message of 3 x nplanes planes (the run's transverse shape)."""
        if self.plane_shape is None:
            raise RuntimeError("SlabRun needs plane_shape=(ny, nx)")
        assert v.size == 3 * nplanes * self.plane_shape[0] * self.plane_shape[1]
        return tuple(self.plane_shape)


class LocalTransport:
    """All slabs of a run in one process: step them in lockstep, handing each phase's messages over."""

    def __init__(self, runs):
        self.runs = list(runs)

    def step(self, n=1):
        for _ in range(n):
            for phase in SlabRun.PHASES:
                for r in self.runs:
                    r.compute(phase)
                outs = [r.outgoing(phase) for r in self.runs]
                for r in self.runs:
                    r.incoming(phase, {q: outs[q][r.rank] for q in r.plan.neighbours(r.rank)})


class DistTransport:
    """One slab per process: each phase's messages go to and come from the neighbouring ranks with
    torch.distributed point-to-point calls (a length, then the float64 payload)."""

    def __init__(self, run: SlabRun):
        import torch.distributed as dist

        if not dist.is_initialized():
            raise RuntimeError("torch.distributed is not initialised")
        self.run, self.dist = run, dist

    def _exchange(self, out):
        import torch

        dist, r = self.dist, self.run
        peers = r.plan.neighbours(r.rank)
        lens = {q: torch.zeros(1, dtype=torch.int64) for q in peers}
        reqs = []
        for q in peers:
            reqs.append(dist.isend(torch.tensor([out[q].size], dtype=torch.int64), dst=q))
            reqs.append(dist.irecv(lens[q], src=q))
        for w in reqs:
            w.wait()
        bufs = {q: torch.empty(int(lens[q].item()), dtype=torch.float64) for q in peers}
        reqs = []
        for q in peers:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(out[q], dtype=np.float64)), dst=q))
            reqs.append(dist.irecv(bufs[q], src=q))
        for w in reqs:
            w.wait()
        return {q: bufs[q].numpy() for q in peers}

    def step(self, n=1):
        r = self.run
        for _ in range(n):
            for phase in SlabRun.PHASES:
                r.compute(phase)
                r.incoming(phase, self._exchange(r.outgoing(phase)))


class LibraryEngine:
    """A library context (paper_0904_0232_gb300.grpic.Simulation) as a slab engine."""

    def __init__(self, sim):
        from . import grpic as G

        self.sim, self.G = sim, G
        self.plane_shape = tuple(sim.shape[1:])
        self._which = {"d": G.GRPIC_FIELD_D, "b": G.GRPIC_FIELD_B, "J": G.GRPIC_FIELD_J}
        self._stages = {"b_half": G.GRPIC_STAGE_B_HALF, "zero_j": G.GRPIC_STAGE_ZERO_J,
                        "push_deposit": G.GRPIC_STAGE_PUSH_DEPOSIT, "b_half2": G.GRPIC_STAGE_B_HALF2,
                        "e": G.GRPIC_STAGE_E, "sort": G.GRPIC_STAGE_SORT}

    def stage(self, name):
        self.sim.stage(self._stages[name])

    def get_planes(self, which, z0, n):
        return self.sim.get_planes(self._which[which], z0, n)

    def set_planes(self, which, z0, planes, add=False):
        self.sim.set_planes(self._which[which], z0, planes, add)

    def get_fields(self):
        return self.sim.get_fields()

    def get_particles(self, s):
        x4, u4, ids = self.sim.get_particles(s)
        return x4, u4, ids

    def load_particles(self, s, q_over_m, q_macro, x4, u4, ids):
        self.sim.load_particles(s, q_over_m, q_macro, x4, u4, ids, umode=self.G.GRPIC_U_FULL)


def library_slab(plan: SlabPlan, rank: int, nx: int, ny: int, m: float, a: float, c: float, dt: float,
                 **sim_kw):
    """A library context for rank `rank`'s planes of the run (nx x ny x plan.nz)."""
    from .grpic import Simulation

    lo, hi = plan.local(rank)
    return Simulation(nx, ny, hi - lo, m, a, c, dt, z_origin=lo, nz_total=plan.nz, **sim_kw)
