"""Serving: runs admitted by the library's server (device-memory budget, slots), resident on
the device, advanced together one batched timestep per tick.

* a run's result is the same alone and in a mix of runs that arrive before and after it
  (J is accumulated with atomics, so within the parity tolerances rather than bitwise);
* a run served in a mix, its plasma generated on the device, matches the oracle started from the
  run's initial state;
* admission waits for memory: with a budget for one run, the second stays queued until the
  first is released;
* requests that could never fit, or that differ in precision, are refused.
"""
import numpy as np
import pytest

import oracle as O
from parity_util import TOL, compare_whole_state, rel_l2
from paper_0904_0232_gb300.grpic import (GRPIC_RUN_DONE, GRPIC_RUN_QUEUED, GRPIC_RUN_RUNNING, GrpicError,
                                         grpic_get_fields, grpic_get_particles, grpic_poll, grpic_request_bytes,
                                         grpic_server_create, grpic_server_destroy, grpic_server_release,
                                         grpic_server_tick, grpic_submit, make_request)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run_to_done(server, ticket, max_ticks=1000):
    for _ in range(max_ticks):
        state, ctx = grpic_poll(server, ticket)
        if state == GRPIC_RUN_DONE:
            return ctx
        grpic_server_tick(server)
    raise AssertionError("run did not finish")


def _snapshot(ctx, n):
    parts = [grpic_get_particles(ctx, s) for s in range(2)]
    return parts, grpic_get_fields(ctx, (n, n, n))


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_same_result_alone_and_in_a_mix(prec):
    A = dict(n=24, m=1.5, a=1.2, ppc=2, nsteps=6, seed=11, precision=prec)
    alone = grpic_server_create(int(4e9), 8)
    ta = grpic_submit(alone, make_request(**A))
    res_alone = _snapshot(_run_to_done(alone, ta), 24)

    mix = grpic_server_create(int(4e9), 8)
    tb = grpic_submit(mix, make_request(n=20, m=1.0, a=0.3, ppc=1, nsteps=3, seed=12, precision=prec))
    grpic_server_tick(mix)
    ta2 = grpic_submit(mix, make_request(**A))
    grpic_server_tick(mix)
    tc = grpic_submit(mix, make_request(n=28, m=2.0, a=1.9, ppc=2, nsteps=10, seed=13, precision=prec))
    res_mix = _snapshot(_run_to_done(mix, ta2), 24)
    for tk in (tb, tc):
        _run_to_done(mix, tk)

    tol = TOL[prec]
    factor = 1.0 if prec == "fp64" else 16.0
    for s in range(2):
        (xa, ua, ia), (xb, ub, ib) = res_alone[0][s], res_mix[0][s]
        oa, ob = np.argsort(ia), np.argsort(ib)
        assert ia.size > 100 and np.array_equal(ia[oa], ib[ob])
        assert np.abs(xa[:3, oa] - xb[:3, ob]).max() <= tol["particles"] * factor * np.abs(xa[:3]).max()
        assert np.abs(ua[:, oa] - ub[:, ob]).max() <= tol["particles"] * factor * np.abs(ua).max()
    (da, ba, Ja), (db, bb, Jb) = res_alone[1], res_mix[1]
    assert rel_l2(Jb, Ja) <= tol["J"] * factor and rel_l2(bb, ba) <= tol["fields"] * factor
    grpic_server_destroy(alone)
    grpic_server_destroy(mix)


@pytest.mark.parametrize("prec,nsteps", [("fp64", 3), ("fp32_mixed", 1)])
def test_served_run_against_oracle(prec, nsteps):
    """The initial state of a run is read from the same request served with no steps (its plasma is
    generated on the device from the seed); the oracle starts from it.  The run itself is served
    in a mix with two others.  FP64: three whole steps, all state compared.  FP32-mixed: one step,
    every particle, and J and the fields off the nodes of zig-zag splits decided within rounding of
    a face (the generated plasma cannot be filtered beforehand)."""
    n = 24
    A = dict(n=n, m=1.5, a=1.2, ppc=2, seed=31, precision=prec)
    s0 = grpic_server_create(int(4e9), 4)
    t0 = grpic_submit(s0, make_request(nsteps=0, **A))
    ctx0 = _run_to_done(s0, t0)
    start = [grpic_get_particles(ctx0, s) for s in range(2)]
    d0, b0, _ = grpic_get_fields(ctx0, (n, n, n))
    grpic_server_destroy(s0)

    req = make_request(nsteps=nsteps, **A)
    ref = O.Oracle(n, n, n, A["m"], A["a"], 1.0, 0.4, threads=0)
    ref.set_fields(d0, b0)
    for s in range(2):
        x, u, ids = start[s]
        ref.load_particles(s, req.q_over_m[s], req.q_macro[s], x, u, ids, umode=0)

    mix = grpic_server_create(int(4e9), 8)
    tb = grpic_submit(mix, make_request(n=20, m=1.0, a=0.3, ppc=1, nsteps=2, seed=32, precision=prec))
    grpic_server_tick(mix)
    ta = grpic_submit(mix, req)
    tc = grpic_submit(mix, make_request(n=28, m=2.0, a=1.9, ppc=1, nsteps=5, seed=33, precision=prec))
    ctx = _run_to_done(mix, ta)
    ref.step(nsteps)

    class View:  # the served context with the comparison helper's accessors
        def get_particles(self, s):
            return grpic_get_particles(ctx, s)

        def get_fields(self):
            return grpic_get_fields(ctx, (n, n, n))

    assert all(start[s][2].size > 100 for s in range(2))
    compare_whole_state(View(), ref, 2, prec, nsteps - 1 if prec == "fp64" else 0, masked=prec != "fp64")
    for tk in (tb, tc):
        _run_to_done(mix, tk)
    grpic_server_destroy(mix)


def test_admission_waits_for_memory():
    req = make_request(n=24, m=1.5, a=0.5, ppc=2, nsteps=4, seed=21)
    one = grpic_request_bytes(req)
    server = grpic_server_create(int(one * 1.5), 8)
    t1 = grpic_submit(server, req)
    t2 = grpic_submit(server, make_request(n=24, m=1.5, a=0.5, ppc=2, nsteps=4, seed=22))
    running, queued = grpic_server_tick(server)
    assert (running, queued) == (1, 1)
    assert grpic_poll(server, t2)[0] == GRPIC_RUN_QUEUED
    _run_to_done(server, t1)
    # finished but not released: its memory is still held, so the second run cannot start
    grpic_server_tick(server)
    assert grpic_poll(server, t2)[0] == GRPIC_RUN_QUEUED
    grpic_server_release(server, t1)
    grpic_server_tick(server)
    assert grpic_poll(server, t2)[0] in (GRPIC_RUN_RUNNING, GRPIC_RUN_DONE)
    _run_to_done(server, t2)
    grpic_server_destroy(server)


def test_refused_requests():
    server = grpic_server_create(int(1e6), 4)
    with pytest.raises(GrpicError) as ei:
        grpic_submit(server, make_request(n=64, m=2.0, a=1.0, ppc=8, nsteps=4, seed=1))
    assert ei.value.code == 8
    grpic_server_destroy(server)
    server = grpic_server_create(int(4e9), 4)
    grpic_submit(server, make_request(n=20, m=1.0, a=0.5, ppc=1, nsteps=2, seed=1, precision="fp32_mixed"))
    with pytest.raises(GrpicError):
        grpic_submit(server, make_request(n=20, m=1.0, a=0.5, ppc=1, nsteps=2, seed=2, precision="fp64"))
    grpic_server_destroy(server)


def test_release_while_others_run():
    """A finished run released at once (its context destroyed) while others keep running: the
    server must not touch the released context again."""
    server = grpic_server_create(int(4e9), 8)
    ta = grpic_submit(server, make_request(n=20, m=1.0, a=0.5, ppc=1, nsteps=2, seed=41))
    tb = grpic_submit(server, make_request(n=24, m=1.5, a=1.0, ppc=1, nsteps=8, seed=42))
    tc = grpic_submit(server, make_request(n=20, m=2.0, a=0.0, ppc=2, nsteps=5, seed=43))
    done = set()
    for _ in range(20):
        grpic_server_tick(server)
        for tk in (ta, tb, tc):
            if tk not in done and grpic_poll(server, tk)[0] == GRPIC_RUN_DONE:
                done.add(tk)
                grpic_server_release(server, tk)
        if len(done) == 3:
            break
    assert done == {ta, tb, tc}
    grpic_server_destroy(server)


def test_unstable_boxes_are_refused():
    """A long run on a box whose faces see f = 2m / R_face > 0.2 is refused with GRPIC_ERR_UNSTABLE
    (the field update grows an edge mode there, independent of the timestep); a short run on the
    same box and a long run on a box four times larger are admitted."""
    from paper_0904_0232_gb300.grpic import GRPIC_ERR_UNSTABLE

    server = grpic_server_create(int(4e9), 8)
    with pytest.raises(GrpicError) as ei:
        grpic_submit(server, make_request(n=32, m=3.0, a=0.0, ppc=1, nsteps=200, seed=51))
    assert ei.value.code == GRPIC_ERR_UNSTABLE
    grpic_submit(server, make_request(n=32, m=3.0, a=0.0, ppc=1, nsteps=50, seed=52))
    grpic_submit(server, make_request(n=128, m=3.0, a=0.0, ppc=1, nsteps=500, seed=53))
    grpic_server_destroy(server)


def test_absorbing_layers_admit_and_complete():
    """The long run refused above, requested with absorbing layers (outer: 4 cells, 0.2 per step at
    the faces; inner: 0.3 per step inside the horizon), is admitted and runs all its steps within
    the step limit, its field staying of the order of the initial one."""
    from paper_0904_0232_gb300.grpic import grpic_get_stats

    server = grpic_server_create(int(4e9), 8)
    req = dict(n=32, m=3.0, a=0.0, ppc=1, nsteps=200, seed=51)
    t = grpic_submit(server, make_request(**req, absorb_inner=0.3, absorb_outer=0.2, absorb_width=4))
    t2 = grpic_submit(server, make_request(**dict(req, a=2.7, seed=54), absorb_inner=0.3, absorb_outer=0.2,
                                           absorb_width=4))
    for tk in (t, t2):
        ctx = _run_to_done(server, tk)
        assert grpic_get_stats(ctx)["steps"] == 200
        d, b, _ = grpic_get_fields(ctx, (32, 32, 32))
        assert np.isfinite(d).all() and np.abs(d).max() < 2.0 and np.abs(b).max() < 2.0, (
            np.abs(d).max(), np.abs(b).max())
        grpic_server_release(server, tk)
    grpic_server_destroy(server)
