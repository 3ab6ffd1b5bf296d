"""Serving loop over GRPIC runs: requests arrive as a Poisson stream, are admitted by the
library's server (device-memory budget and slots), run together in batched timesteps while
resident on the device, and their completion latency is recorded.

    python -m paper_0904_0232_gb300.serve --rate 5 --duration 20
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .grpic import (GRPIC_RUN_DONE, grpic_get_stats, grpic_poll, grpic_request_bytes, grpic_server_create,
                    grpic_server_destroy, grpic_server_release, grpic_server_tick, grpic_submit, make_request)


def sample_requests(n, seed, grids=(32, 48, 64), ppc=(1, 8), steps=(50, 200), m=(1.0, 4.0), spin_max=0.99):
    """n request specs drawn from the stated ranges (grid, particles per cell per species,
    timesteps, mass in cells, spin in units of m)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        g = int(rng.choice(grids))
        mm = float(rng.uniform(*m))
        out.append(dict(n=g, m=mm, a=float(rng.uniform(0.0, spin_max)) * mm, ppc=int(rng.integers(ppc[0], ppc[1] + 1)),
                        nsteps=int(rng.integers(steps[0], steps[1] + 1)), seed=1000 + k))
    return out


def serve_poisson(rate, duration, budget_bytes, slots, seed=0, max_wall=None, **spec_ranges):
    """Run a Poisson arrival stream (rate per second over `duration` seconds of arrivals) to
    completion.  Returns latencies (s), aggregate particle-steps/s and counts."""
    rng = np.random.default_rng(seed)
    arrivals = []
    t = rng.exponential(1.0 / rate)
    while t < duration:
        arrivals.append(t)
        t += rng.exponential(1.0 / rate)
    specs = sample_requests(len(arrivals), seed + 1, **spec_ranges)
    server = grpic_server_create(budget_bytes, slots)
    pending = {}   # ticket -> arrival time
    lat = []
    psteps = 0
    nxt = 0
    t0 = time.perf_counter()
    try:
        while nxt < len(arrivals) or pending:
            now = time.perf_counter() - t0
            if max_wall is not None and now > max_wall:
                break
            while nxt < len(arrivals) and arrivals[nxt] <= now:
                req = make_request(**specs[nxt])
                pending[grpic_submit(server, req)] = arrivals[nxt]
                nxt += 1
            if pending:
                grpic_server_tick(server)
                done_now = time.perf_counter() - t0
                for tk in list(pending):
                    state, ctx = grpic_poll(server, tk)
                    if state == GRPIC_RUN_DONE:
                        psteps += grpic_get_stats(ctx)["particle_steps"]
                        lat.append(done_now - pending.pop(tk))
                        grpic_server_release(server, tk)
            else:
                time.sleep(min(0.001, max(0.0, arrivals[nxt] - now)) if nxt < len(arrivals) else 0)
        wall = time.perf_counter() - t0
    finally:
        grpic_server_destroy(server)
    lat = np.array(lat)
    return {"rate": rate, "arrivals": len(arrivals), "completed": int(lat.size),
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "particle_steps_per_s": psteps / wall if wall > 0 else 0.0, "wall_s": wall}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--rate", type=float, nargs="+", default=[2.0])
    p.add_argument("--duration", type=float, default=10.0)
    p.add_argument("--budget-gb", type=float, default=100.0)
    p.add_argument("--slots", type=int, default=64)
    args = p.parse_args()
    for r in args.rate:
        print(json.dumps(serve_poisson(r, args.duration, int(args.budget_gb * 1e9), args.slots)), flush=True)


if __name__ == "__main__":
    main()
