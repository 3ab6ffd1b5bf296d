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

from .grpic import (GRPIC_OK, GRPIC_RUN_DONE, STATUS_NAMES, GrpicError, grpic_get_invariants, grpic_get_stats,
                    grpic_poll, grpic_request_bytes, grpic_server_create, grpic_server_destroy,
                    grpic_server_release, grpic_server_tick, grpic_submit, make_request)


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


def layers_for(n):
    """Absorbing layers a client requests for an n^3 box: 0.3 per step inside the horizon, 0.2 per
    step at the faces over n/8 cells (4 to 8).  Without them, long runs on boxes whose faces see
    f = 2m / R_face > 0.2 are refused (a mode grows at the frozen faces there)."""
    return dict(absorb_inner=0.3, absorb_outer=0.2, absorb_width=int(min(8, max(4, n // 8))))


def serve_poisson(rate, duration, budget_bytes, slots, seed=0, max_wall=None, layers=True, **spec_ranges):
    """Run a Poisson arrival stream (rate per second over `duration` seconds of arrivals) to
    completion, every request with absorbing layers unless `layers` is false.  Returns latencies
    (s), aggregate particle-steps/s and counts."""
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
    failed = []
    refused = []
    inv = []   # per finished run: |g(u,u) + c^2| / c^2 at the end and the E, L changes over the run
    psteps = 0
    nxt = 0
    t0 = time.perf_counter()
    try:
        while nxt < len(arrivals) or pending:
            now = time.perf_counter() - t0
            if max_wall is not None and now > max_wall:
                break
            while nxt < len(arrivals) and arrivals[nxt] <= now:
                spec = specs[nxt]
                req = make_request(**spec, **(layers_for(spec["n"]) if layers else {}))
                try:
                    pending[grpic_submit(server, req)] = arrivals[nxt]
                except GrpicError as e:  # refused at admission (e.g. GRPIC_ERR_UNSTABLE), with its reason
                    refused.append(STATUS_NAMES.get(e.code, e.code))
                nxt += 1
            if pending:
                grpic_server_tick(server)
                done_now = time.perf_counter() - t0
                for tk in list(pending):
                    state, ctx, status = grpic_poll(server, tk, with_status=True)
                    if state == GRPIC_RUN_DONE:
                        if ctx:
                            psteps += grpic_get_stats(ctx)["particle_steps"]
                            iv = grpic_get_invariants(ctx)
                            inv.append((iv["norm_max"], iv["energy_max"], iv["angmom_max"]))
                        if status == GRPIC_OK:
                            lat.append(done_now - pending.pop(tk))
                        else:
                            failed.append(STATUS_NAMES.get(status, status))
                            pending.pop(tk)
                        grpic_server_release(server, tk)
            else:
                time.sleep(min(0.001, max(0.0, arrivals[nxt] - now)) if nxt < len(arrivals) else 0)
        wall = time.perf_counter() - t0
    finally:
        grpic_server_destroy(server)
    lat = np.array(lat)
    # runs still queued or running when the wall-clock bound stopped the loop: their latency is
    # at least (end - arrival), and arrivals not yet submitted count from their arrival time
    cens = np.array([wall - a for a in pending.values()] + [wall - a for a in arrivals[nxt:] if a <= wall])
    allv = np.concatenate([lat, cens]) if cens.size else lat
    return {"rate": rate, "arrivals": len(arrivals), "completed": int(lat.size), "unfinished": int(cens.size),
            "failed": len(failed), "failed_status": sorted(set(failed)),
            "refused": len(refused), "refused_status": sorted(set(refused)),
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "p50_s_lower_bound_all": float(np.percentile(allv, 50)) if allv.size else None,
            "p99_s_lower_bound_all": float(np.percentile(allv, 99)) if allv.size else None,
            "particle_steps_per_s": psteps / wall if wall > 0 else 0.0, "wall_s": wall,
            "invariants": ({"runs": len(inv), "norm_max": max(v[0] for v in inv),
                            "norm_max_median_run": float(np.median([v[0] for v in inv])),
                            "energy_change_max_median_run": float(np.median([v[1] for v in inv])),
                            "angmom_change_max_median_run": float(np.median([v[2] for v in inv])),
                            "note": "per run, from its initial plasma to its end: |g(u,u)+c^2|/c^2 (Eq. 7) "
                                    "and the changes of -u_4 and u_phi over the tracked subsample, /c"}
                           if inv else None)}


# Request mixes: grid edge, particles per cell per species, timesteps (each drawn uniformly), with
# m in [1, 4] cells and a in [0, 0.99] m.  "full": the serving configuration's ranges; "light": a
# mix one GPU serves without a growing queue at a few requests per second.
MIXES = {
    "full": dict(grids=(32, 48, 64, 96, 128), ppc=(1, 64), steps=(50, 500)),
    "light": dict(grids=(32, 48, 64), ppc=(1, 8), steps=(50, 200)),
}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--rate", type=float, nargs="+", default=[2.0])
    p.add_argument("--duration", type=float, default=10.0, help="seconds of Poisson arrivals per rate")
    p.add_argument("--mix", choices=sorted(MIXES), default="light")
    p.add_argument("--budget-gb", type=float, default=100.0)
    p.add_argument("--slots", type=int, default=64)
    p.add_argument("--max-wall", type=float, default=None, help="stop waiting for completions after this")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-layers", action="store_true", help="requests without absorbing layers")
    args = p.parse_args()
    for r in args.rate:
        res = serve_poisson(r, args.duration, int(args.budget_gb * 1e9), args.slots, seed=args.seed,
                            max_wall=args.max_wall, layers=not args.no_layers, **MIXES[args.mix])
        res.update(mix=args.mix, mix_ranges=MIXES[args.mix], budget_gb=args.budget_gb, slots=args.slots,
                   arrival_window_s=args.duration, absorbing_layers=not args.no_layers)
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
