"""Absorbing layers on the device (relaxation toward the field as last set, after the second B
half-step and the E step; an inner layer inside the horizon, an outer one next to the frozen faces).

* whole steps with both layers against the oracle, for one context and for the batched engine;
* the growing mode they are there for: a vacuum run with a rapidly rotating hole resolved by
  m = 8 cells, whose field near the horizon grows by orders of magnitude over 500 steps with the
  inside of the horizon frozen, stays of the order of the initial field with the layers.
"""
import numpy as np
import pytest

from parity_util import compare_whole_state, gpu_from_oracle, oracle_start, well_conditioned
from paper_0904_0232_gb300 import synth
from paper_0904_0232_gb300.grpic import Simulation, grpic_batch_create, grpic_batch_destroy, grpic_batch_step

pytestmark = pytest.mark.gpu

LAYERS = dict(absorb_inner=0.3, absorb_outer=0.25, absorb_width=4)


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _workload(seed, n=24, m=2.5, am=0.9):
    return synth.plasma(f"absorb{seed}", n, m, am * m, 1.0, 0.4, 0.1, 3, 2, (-1.0, 1.0), 0.1, seed=seed,
                        r_min=1.5 * m)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_layers_against_oracle(prec):
    """Three whole steps of a pair plasma around a = 0.9m (m = 2.5) on a 24^3 grid with both layers
    (the inner one covers r_+/2 <= r < r_+, the outer one the four cells next to the faces): every
    particle, J node and field value after every step against the oracle."""
    wl = well_conditioned(_workload(5), 3, threads=0, **LAYERS)
    ref = oracle_start(wl, **LAYERS)
    sim = gpu_from_oracle(ref, wl, prec, **LAYERS)
    rec = []
    for step in range(3):
        sim.step(1)
        ref.step(1)
        compare_whole_state(sim, ref, len(wl.species), prec, step, rec)
    print("layers vs oracle", prec, max(r[2] for r in rec if r[1] == "J,b,d"))


def test_batched_layers_against_oracle():
    """The batched field launches apply each instance's own layers: one instance with both layers,
    one with the outer layer only, one without, three whole steps against the oracle."""
    cfgs = [LAYERS, dict(absorb_outer=0.4, absorb_width=3), {}]
    wls = [well_conditioned(_workload(20 + k, n=20 + 4 * k, m=1.5 + 0.5 * k), 3, threads=0, **cfg)
           for k, cfg in enumerate(cfgs)]
    refs = [oracle_start(w, **cfg) for w, cfg in zip(wls, cfgs)]
    sims = [gpu_from_oracle(r, w, "fp32_mixed", **cfg) for r, w, cfg in zip(refs, wls, cfgs)]
    b = grpic_batch_create([s.handle for s in sims])
    rec = []
    for step in range(3):
        grpic_batch_step(b, 1)
        for r in refs:
            r.step(1)
        for sim, ref, wl in zip(sims, refs, wls):
            compare_whole_state(sim, ref, len(wl.species), "fp32_mixed", step, rec)
    grpic_batch_destroy(b)


def _vacuum_peak(layers, n=192, m=8.0, am=0.95, steps=500):
    sim = Simulation(n, n, n, m, am * m, 1.0, 0.4, precision="fp32_mixed", **layers)
    sim.set_uniform_field(B=(0.0, 0.0, 0.1))
    sim.step(steps)
    d, b, _ = sim.get_fields()
    sim.close()
    return float(np.sqrt((d ** 2).sum(0)).max()), float(np.abs(b).max())


def test_layers_hold_the_near_horizon_mode():
    """a = 0.95m with m = 8 cells, B_z = 0.1, 500 steps: with the inside of the horizon frozen the
    field next to the horizon grows past 1e3 (it e-folds about every 40 steps); with the layers it
    stays below 5 (the Wald-like field near the hole is of order 1 here)."""
    frozen, _ = _vacuum_peak({})
    absorbed, bmax = _vacuum_peak(dict(absorb_inner=0.3, absorb_outer=0.2, absorb_width=12))
    print("near-horizon mode: frozen", frozen, "layers", absorbed, bmax)
    assert frozen > 1e3
    assert absorbed < 5.0 and bmax < 5.0
