"""The FP32-mixed push with a far-field code path: particles within r_fp64 + |a| + 4 cells of the
hole ("near") take the FP32-mixed code with the FP64 policy, the others FP32-only code -- either
per warp in one kernel (split = 0) or in separate near-hole and far-field kernels on two streams
(split = 1).

* against the oracle, on a grid where both populations are present;
* against the single mixed kernel (GRPIC_SINGLE_PUSH_KERNEL): the same particle-step, the same
  number of FP64 evaluations (no far particle ever needed one);
* every launch-shape choice of grpic_tuning gives the same result;
* the FP64 reciprocal / quotient / root of the near-hole evaluations against the IEEE operations.
"""
import numpy as np
import pytest

from parity_util import TOL, check_j, gpu_from_oracle, oracle_start, particle_errors, rel_l2, small_kerr
from paper_0904_0232_gb300.grpic import (GRPIC_SINGLE_PUSH_KERNEL, GRPIC_STAGE_PUSH_DEPOSIT, GRPIC_STAGE_SORT,
                                         GRPIC_STAGE_ZERO_J,
                                         GrpicError, grpic_check_conversions, grpic_check_newton64)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


M, A, N = 1.5, 1.2, 40
R_NEAR = 4.0 * M + abs(A) + 4.0


def _workload(seed=31):
    wl = small_kerr(n=N, ppc=1, seed=seed, m=M, a=A, r_min=1.6 * M)
    cen = (N - 1) / 2.0
    R = np.concatenate([np.sqrt(((sp.x4[:3] - cen) ** 2).sum(0)) for sp in wl.species])
    near = int((R < R_NEAR).sum())
    assert 0.02 * R.size < near < 0.5 * R.size  # both kernels have work
    return wl


def _push_once(sim):
    sim.stage(GRPIC_STAGE_ZERO_J)
    sim.stage(GRPIC_STAGE_PUSH_DEPOSIT)


def _state(sim):
    out = []
    for s in range(2):
        x, u, ids = sim.get_particles(s)
        o = np.argsort(ids)
        out.append((x[:, o], u[:, o], ids[o]))
    return out, sim.get_fields()[2], sim.stats()


@pytest.mark.parametrize("mode", [0, 1])
def test_split_push_against_oracle(mode):
    wl = _workload()
    ref = oracle_start(wl)
    sim = gpu_from_oracle(ref, wl, "fp32_mixed")
    sim.set_tuning(split=mode)
    n_live = sum(sim.num_particles(s) for s in range(2))
    ref.zero_j()
    ref.push_deposit()
    _push_once(sim)
    assert sim.stats()["particle_steps"] == n_live  # each particle pushed once, by one of the two kernels
    _, _, J = sim.get_fields()
    sim.stage(GRPIC_STAGE_SORT)  # drop the particles this push removed, as the oracle has
    tol = TOL["fp32_mixed"]
    for s in range(2):
        ex, e4, eu = particle_errors(sim, ref, s)
        assert max(ex, e4, eu) <= tol["particles"], (s, ex, e4, eu)
    _, _, Jr = ref.get_fields()
    check_j(J, Jr, ref, 2, "fp32_mixed")  # 1e-5 off the nodes of splits decided within rounding of a face
    assert sim.stats()["fp64_evals"] > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_split_equals_single_kernel(mode):
    wl = _workload(seed=32)
    ref = oracle_start(wl)
    split = gpu_from_oracle(ref, wl, "fp32_mixed")
    split.set_tuning(split=mode)
    single = gpu_from_oracle(ref, wl, "fp32_mixed", flags=GRPIC_SINGLE_PUSH_KERNEL)
    _push_once(split)
    _push_once(single)
    (ps, Js, sts), (pq, Jq, stq) = _state(split), _state(single)
    assert sts["fp64_evals"] == stq["fp64_evals"] > 0
    assert sts["particle_steps"] == stq["particle_steps"]
    for (xs, us, i_s), (xq, uq, iq) in zip(ps, pq):
        assert np.array_equal(i_s, iq)
        assert np.abs(xs - xq).max() <= 1e-6 * np.abs(xq).max()
        assert np.abs(us - uq).max() <= 1e-6 * np.abs(uq).max()
    # the two kernels compile the same FP32 arithmetic separately (contraction may differ in
    # the last bit) and accumulate J in another order
    assert rel_l2(Js, Jq) <= 1e-6
    # whole steps stay together too
    split.step(4)
    single.step(4)
    (ps, Js, _), (pq, Jq, _) = _state(split), _state(single)
    for (xs, us, i_s), (xq, uq, iq) in zip(ps, pq):
        assert np.array_equal(i_s, iq)
        assert np.abs(xs - xq).max() <= 1e-5 * np.abs(xq).max()


@pytest.mark.parametrize("far,near,overlap,split,j_tile,spread,table", [
    (4, 1, 1, 1, 0, 0, 0), (5, 2, 0, 1, 0, 0, 0), (6, 3, 1, 1, 0, 0, 0), (5, 4, 0, 1, 0, 0, 0),
    (4, 4, 1, 0, 0, 0, 0), (5, 4, 1, 0, 0, 0, 0), (4, 4, 1, 0, 1, 0, 0), (5, 4, 1, 0, 1, 0, 0),
    (4, 4, 1, 0, 0, 1, 0), (5, 4, 1, 0, 1, 1, 0), (4, 4, 1, 0, 0, 4, 0), (4, 4, 1, 0, 0, 16, 0),
    (5, 4, 1, 0, 1, 64, 0), (4, 4, 1, 0, 0, 16, 1), (5, 4, 1, 0, 0, 1, 1)])
def test_tuning_variants_agree(far, near, overlap, split, j_tile, spread, table):
    wl = _workload(seed=33)
    ref = oracle_start(wl)
    base = gpu_from_oracle(ref, wl, "fp32_mixed", flags=GRPIC_SINGLE_PUSH_KERNEL)
    var = gpu_from_oracle(ref, wl, "fp32_mixed")
    var.set_tuning(far_min_blocks=far, near_blocks_per_sm=near, sort_interval=1, overlap=overlap, split=split,
                   j_tile=j_tile, spread=spread, area_table=table)
    assert var.tuning() == dict(far_min_blocks=far, near_blocks_per_sm=near, sort_interval=1, overlap=overlap,
                                split=split, j_tile=j_tile, spread=spread, area_table=table)
    _push_once(base)
    _push_once(var)
    (pb, Jb, sb), (pv, Jv, sv) = _state(base), _state(var)
    assert sb["fp64_evals"] == sv["fp64_evals"]
    for (xb, ub, ib), (xv, uv, iv) in zip(pb, pv):
        assert np.array_equal(ib, iv)
        assert np.abs(xb - xv).max() <= 1e-6 * np.abs(xb).max()
        assert np.abs(ub - uv).max() <= 1e-6 * np.abs(ub).max()
    assert sb["particle_steps"] == sv["particle_steps"]
    assert rel_l2(Jv, Jb) <= 1e-6


def test_sort_interval_from_tuning_matches_oracle():
    wl = _workload(seed=34)
    ref = oracle_start(wl)
    sim = gpu_from_oracle(ref, wl, "fp32_mixed")
    sim.set_tuning(far_min_blocks=5, near_blocks_per_sm=2, sort_interval=3, overlap=1)
    ref.step(2)
    sim.step(2)
    tol = TOL["fp32_mixed"]
    for s in range(2):
        ex, e4, eu = particle_errors(sim, ref, s)
        assert max(ex, eu) <= tol["particles"] * 8, (s, ex, eu)


def test_fresh_contexts_push_each_particle_once():
    """The near kernel runs concurrently with the far kernel; neither may push a particle the
    other owns, whichever starts first (fresh contexts, first launches included)."""
    wl = _workload(seed=36)
    ref = oracle_start(wl)
    single = gpu_from_oracle(ref, wl, "fp32_mixed", flags=GRPIC_SINGLE_PUSH_KERNEL)
    _push_once(single)
    single.step(2)
    want = single.stats()
    single.close()
    for rep in range(4):
        sim = gpu_from_oracle(ref, wl, "fp32_mixed")
        sim.set_tuning(far_min_blocks=4 + rep // 2, near_blocks_per_sm=1 + rep, sort_interval=1, overlap=rep // 2,
                       split=rep % 2)
        n_live = sum(sim.num_particles(s) for s in range(2))
        _push_once(sim)
        assert sim.stats()["particle_steps"] == n_live, rep
        sim.step(2)
        got = sim.stats()
        assert got["particle_steps"] == want["particle_steps"], rep
        assert got["removed_horizon"] == want["removed_horizon"], rep
        sim.close()


def test_tuning_validation():
    wl = _workload(seed=35)
    ref = oracle_start(wl)
    sim = gpu_from_oracle(ref, wl, "fp32_mixed")
    for bad in [(3, 2, 1, 1, 0), (7, 2, 1, 1, 0), (5, 0, 1, 1, 0), (5, 2, 0, 1, 0), (5, 2, 1, 2, 0), (5, 2, 1, 1, 2),
                (5, 2, 1, 1, 0, 2), (5, 2, 1, 1, 0, 0, 3), (5, 2, 1, 1, 0, 0, 128), (5, 2, 1, 1, 0, 0, -1)]:
        with pytest.raises(GrpicError):
            sim.set_tuning(*bad)
    assert sim.tuning()["far_min_blocks"] == 4


def test_seeded_fp64_ops_against_ieee():
    # one Newton step from an FP32 estimate (relative error a few 2^-23) squares that error
    err = grpic_check_newton64(1 << 22)
    print("SeededOps64 max relative deviation from IEEE:", err)
    assert max(err.values()) <= 1e-12


def test_integer_conversions_match_hardware():
    bad = grpic_check_conversions(1 << 24)
    assert bad == dict(widen=0, narrow=0)


def test_j_tile_against_oracle_and_over_steps():
    wl = _workload(seed=37)
    ref = oracle_start(wl)
    sim = gpu_from_oracle(ref, wl, "fp32_mixed")
    sim.set_tuning(j_tile=1)
    plain = gpu_from_oracle(ref, wl, "fp32_mixed")
    ref.zero_j()
    ref.push_deposit()
    _push_once(sim)
    _push_once(plain)
    _, _, J = sim.get_fields()
    _, _, Jr = ref.get_fields()
    _, _, Jp = plain.get_fields()
    assert rel_l2(J, Jr) <= TOL["fp32_mixed"]["J"] * 10
    # FP32 partial sums per block instead of one FP64 add per contribution: within FP32 rounding
    assert rel_l2(J, Jp) <= 1e-6
    sim.step(3)
    plain.step(3)
    (ps, Js, _), (pp, Jq, _) = _state(sim), _state(plain)
    for (xs, us, i_s), (xq, uq, iq) in zip(ps, pp):
        assert np.array_equal(i_s, iq)
        assert np.abs(xs - xq).max() <= 1e-5 * np.abs(xq).max()
