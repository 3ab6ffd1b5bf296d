"""Parity at the largest configuration's full size: Kerr a = 0.95 m, m = 8, 384^3, an accretion
disk inside a corona, ~1e9 particles in FP32-mixed (generated on the device), pushed by the
library in the launch configuration the context uses; a strided sample of ~25 k particles per
species is pushed one by one by the oracle from the same start, after the oracle's own first B
half-step on the whole 384^3 grid.  Compared: every sampled particle's position after the push
(removed ones included) and the velocities of the survivors, at the FP32 tolerance.

Needs ~170 GB of device memory (particle buffers, generation and read-back staging) and ~12 GB
of host memory for the oracle's fields; skipped where the device has less free memory.
"""
import numpy as np
import pytest

import oracle as O
from parity_util import TOL
from paper_0904_0232_gb300 import synth_disk
from paper_0904_0232_gb300.grpic import GRPIC_STAGE_B_HALF, GRPIC_STAGE_PUSH_DEPOSIT, GRPIC_STAGE_ZERO_J, Simulation

pytestmark = pytest.mark.gpu


def test_disk_corona_384_sampled():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 170e9:
        pytest.skip("needs ~170 GB of free device memory")
    wl = synth_disk.kerr_disk_corona(n=384, seed=3)
    assert 0.9e9 < wl.n_particles < 1.1e9
    samples = []
    for sp in wl.species:
        n = sp.ids.numel()
        sel = torch.arange(0, n, max(1, n // 25000), device=sp.ids.device)
        samples.append((sp.x4[:, sel].cpu().numpy(), sp.u4[:3, sel].cpu().numpy(),
                        sp.ids[sel].cpu().numpy().astype(np.uint32)))
    sim = Simulation(wl.n, wl.n, wl.n, wl.m, wl.a, wl.c, wl.dt, precision="fp32_mixed")
    sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
    meta = [(sp.q_over_m, sp.q_macro, sp.umode) for sp in wl.species]
    geo = (wl.n, wl.m, wl.a, wl.c, wl.dt, wl.B0)
    for s, sp in enumerate(wl.species):
        sim.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.u4, sp.ids, umode=sp.umode)
    del wl, sp
    torch.cuda.empty_cache()
    sim.stage(GRPIC_STAGE_B_HALF)
    sim.stage(GRPIC_STAGE_ZERO_J)
    sim.stage(GRPIC_STAGE_PUSH_DEPOSIT)
    assert sim.stats()["fp64_evals"] > 0
    got = []
    for s, (_, _, sid) in enumerate(samples):
        x, u, ids = sim.get_particles(s, device=True)
        pick = torch.isin(ids, torch.from_numpy(sid.astype(np.int32)).cuda())
        xs, us, i_s = x[:, pick].cpu().numpy(), u[:, pick].cpu().numpy(), ids[pick].cpu().numpy().astype(np.uint32)
        o = np.argsort(i_s)
        got.append((xs[:, o], us[:, o], i_s[o]))
        del x, u, ids, pick
        torch.cuda.empty_cache()
    sim.close()

    n, m, a, c, dt, B0 = geo
    ref = O.Oracle(n, n, n, m, a, c, dt, threads=4, flags=O.NO_GAMMA_TERMS)
    ref.init_uniform_field(B=(0.0, 0.0, B0))
    ref.b_half()
    for s, ((x4, usp, ids), (qm, qmac, umode)) in enumerate(zip(samples, meta)):
        ref.load_particles(s, qm, qmac, x4, usp, ids, umode=umode)
    ref.push_deposit()
    tol = TOL["fp32_mixed"]["particles"]
    for s in range(len(samples)):
        xr0, xr1, ir = ref.last_moves(s)
        x1, u1, i1 = got[s]
        # the oracle drops particles inside r_+ at load as the library does: same ids
        assert np.array_equal(ir, i1)
        ex = np.abs(x1[:3] - xr1).max(0) / np.abs(xr1).max(0)
        assert ex.max() <= tol, (s, ex.max())
        xs, us, ids_s = ref.get_particles(s)
        keep = np.searchsorted(i1, ids_s)
        eu = np.abs(u1[:, keep] - us).max(0) / np.abs(us).max(0)
        assert eu.max() <= tol, (s, eu.max())

