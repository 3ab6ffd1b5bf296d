"""Whole-cycle behaviour of the oracle: removal at the horizon and the outer boundary (A15),
the step-size check (A17), determinism across thread counts, and a regression snapshot."""
import os
import sys

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))


def test_horizon_and_outer_removal():
    N, m, a = 20, 2.0, 1.0
    o = O.Oracle(N, N, N, m, a, 1.0, 0.4, flags=O.FROZEN_FIELDS)
    Xc = o.centre
    rp = o.r_plus
    # 0: just outside the horizon falling in fast; 1: next to the outer boundary moving out;
    # 2: at rest far away (stays)
    x4 = np.array([[Xc[0] + rp + 0.05, 18.0, Xc[0] + 6.0],
                   [Xc[1], Xc[1], Xc[1]],
                   [Xc[2], Xc[2], Xc[2] + 3.0],
                   [0.0, 0.0, 0.0]])
    u = np.zeros((4, 3))
    u[:3, 0] = (-0.8, 0.0, 0.0)
    u[:3, 1] = (0.9, 0.0, 0.0)
    for p in range(3):
        u[:, p] = O.solve_u4(x4[:3, p] - Xc, m, a, 1.0, u[:3, p], 1)
    o.load_particles(0, 0.0, 0.0, x4, u, [0, 1, 2])
    o.step(1)
    st = o.stats()
    assert st["removed_horizon"] == 1 and st["removed_outer"] == 1
    assert list(o.get_particles(0)[2]) == [2]


def test_step_limit_is_an_error():
    """A move of a full cell or more in one step is refused (Umeda's split needs < 1 cell)."""
    N = 16
    o = O.Oracle(N, N, N, 0.0, 0.0, 1.0, 1.2, flags=O.FROZEN_FIELDS)
    x4 = np.array([[7.0], [7.0], [7.0], [0.0]])
    u = np.array([[5.0], [0.0], [0.0], [np.sqrt(26.0)]])
    o.load_particles(0, 0.0, 0.0, x4, u, [0])
    with pytest.raises(O.OracleError) as ei:
        o.step(1)
    assert ei.value.code == O.ERR_CFL


def test_load_rejects_positions_outside_domain():
    o = O.Oracle(12, 12, 12, 0.0, 0.0, 1.0, 0.4)
    with pytest.raises(O.OracleError):
        o.load_particles(0, 1.0, 0.0, np.array([[0.5], [5.0], [5.0], [0.0]]), np.array([[0.0], [0.0], [0.0], [1.0]]), [0])


def test_thread_count_changes_only_rounding():
    """Per-thread J copies are reduced in a fixed order: results differ only in rounding."""
    import make_oracle_golden as G

    runs = []
    for t in (1, 3):
        o = G.tiny_case(threads=t)
        o.step(2)
        runs.append(o.get_fields())
    (d1, b1, J1), (d3, b3, J3) = runs
    assert np.abs(J3 - J1).max() <= 1e-14 * np.abs(J1).max()
    assert np.abs(d3 - d1).max() <= 1e-14 * np.abs(d1).max()
    assert np.abs(b3 - b1).max() <= 1e-14 * np.abs(b1).max()


def test_regression_snapshot():
    import make_oracle_golden as G

    gold = np.load(os.path.join(HERE, "golden", "oracle_tiny_step.npz"))
    out = G.run()
    for k in gold.files:
        assert out[k].shape == gold[k].shape
        assert np.allclose(out[k], gold[k], rtol=1e-13, atol=1e-15), k


def test_particles_inside_horizon_are_dropped_at_load():
    """The removal rule r <= r_+ (A15) applies from the start."""
    N, m, a = 20, 2.0, 1.0
    o = O.Oracle(N, N, N, m, a, 1.0, 0.4)
    Xc = o.centre
    x4 = np.array([[Xc[0] + 0.3, Xc[0] + 7.0], [Xc[1], Xc[1]], [Xc[2] + 0.2, Xc[2]], [0.0, 0.0]])
    o.load_particles(0, -1.0, 0.0, x4, np.zeros((3, 2)), [5, 6], umode=1)
    assert list(o.get_particles(0)[2]) == [6]
    assert o.stats()["removed_horizon"] == 1
