"""The operation count of a particle-step (oracle/flop_count.py) belongs to arithmetic that
produces the method's result: its particle-step -- RK4 push with Eq. 16, CIC gather, Eq. 8 and
Eq. 15 at the particle, Umeda's split with the Eq. 18 weights -- equals the oracle's, particle
state and every J contribution, to rounding.  The counts per quadrature order are those stored
in tests/golden/flop_count.json (written by tests/golden/make_flop_count.py)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import flop_count as FC
from paper_0904_0232_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _setup(n=16, m=2.0, a=1.6, seed=3):
    rng = np.random.default_rng(seed)
    d, b = synth.random_fields((n, n, n), seed, 0.05)
    cen = (n - 1) / 2.0
    pts = []
    while len(pts) < 12:
        x = rng.uniform(2.0, n - 3.0, 3)
        if np.linalg.norm(x - cen) > 2.5 * m:
            pts.append(x)
    return n, m, a, d, b, pts, rng


@pytest.mark.parametrize("Q", [1, 2, 3])
def test_counted_step_equals_oracle(Q):
    n, m, a, d, b, pts, rng = _setup()
    run = FC.Run((n, n, n), m, a, 1.0, 0.4, Q)
    fields = list(d) + list(b)
    for k, x in enumerate(pts):
        usp = rng.normal(0, 0.3, 3)
        u = O.solve_u4(x - (n - 1) / 2.0, m, a, 1.0, usp, 2)
        qm, qmac = (-1.0, 0.01) if k % 2 else (0.05, 0.02)
        o = O.Oracle(n, n, n, m, a, 1.0, 0.4, quad_order=Q, flags=O.FROZEN_FIELDS)
        o.set_fields(d, b)
        o.load_particles(0, qm, qmac, np.r_[x, 0.0].reshape(4, 1), u.reshape(4, 1), [k], umode=0)
        o.zero_j()
        o.push_deposit()
        xo, uo, _ = o.get_particles(0)
        Jo = o.get_fields()[2]
        nops, (x1, u1, J, removed) = FC.count_step(run, fields, np.r_[x, 0.0], u, qm, qmac)
        assert not removed and xo.shape[1] == 1
        assert np.allclose(x1, xo[:, 0], rtol=1e-13, atol=1e-13)
        assert np.allclose(u1, uo[:, 0], rtol=1e-12, atol=1e-14)
        Jc = np.zeros_like(Jo)
        for (K, kk, jj, ii), v in J.items():
            Jc[K, kk, jj, ii] += v
        assert np.abs(Jc - Jo).max() <= 1e-13 * np.abs(Jo).max()
        assert nops > 0


def test_counts_are_the_stored_ones():
    with open(os.path.join(HERE, "golden", "flop_count.json")) as fh:
        stored = json.load(fh)
    n, m, a, d, b, pts, rng = _setup()
    fields = list(d) + list(b)
    for Q in (1, 2, 3):
        run = FC.Run((n, n, n), m, a, 1.0, 0.4, Q)
        counts = []
        for k, x in enumerate(pts):
            u = O.solve_u4(x - (n - 1) / 2.0, m, a, 1.0, rng.normal(0, 0.3, 3), 2)
            counts.append(FC.count_step(run, fields, np.r_[x, 0.0], u, -1.0, 0.01)[0])
        assert max(counts) - min(counts) <= 0.02 * np.mean(counts)
        assert abs(np.mean(counts) - stored["ops_per_particle_step"][str(Q)]) <= 0.02 * np.mean(counts)
