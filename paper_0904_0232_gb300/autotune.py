"""Autotuner for the launch-shape choices of a GRPIC context (grpic_tuning in include/grpic.h):
whether the FP32-mixed push runs as one kernel with a per-warp choice of code or split into
near-hole and far-field kernels, the register budget of the far-field code (resident blocks
per SM), the persistent blocks per SM of the near-hole kernel, whether that kernel overlaps the
far one on a second stream, whether the per-warp kernel accumulates J in shared-memory tiles,
whether its far-field warps take the face areas from per-cell fits, and the sort interval.

Coordinate descent: starting from the current choice, each knob in turn is set to each of its
values while the others stay fixed, and the fastest is kept; two rounds.  A trial times
`steps` whole timesteps with CUDA events on the context's stream after one untimed step (the
first step after a change of sort interval or kernel variant pays for the change).  Trials
advance the simulation like warm-up steps do, and the step time drifts as the state evolves (the
FP64 load grows as plasma falls in), so each value of a knob is timed twice, the values in
forward and then in reverse order, and the means are compared: a steady drift cancels.  A
combination the context refuses (GrpicError: the area fits with a J tile, say) is timed with one
other knob back at its first choice instead, or skipped.  Winners are cached in a JSON file keyed by the
device name and a workload signature, so later runs can reuse them without tuning.

The batched engine has one knob, the persistent blocks per SM of its launches; tune_batch
times whole batched steps for each value.
"""
from __future__ import annotations

import json
import os

from .grpic import GrpicError

CHOICES = {
    "split": (0, 1),
    "spread": (0, 1, 16),
    "j_tile": (0, 1),
    "area_table": (0, 1),
    "far_min_blocks": (4, 5, 6),
    "near_blocks_per_sm": (1, 2, 4),
    "overlap": (0, 1),
    "sort_interval": (1, 2, 4),
}
BATCH_CHOICES = (4, 8, 16)
DEFAULT_CACHE = os.environ.get("GRPIC_TUNE_CACHE",
                               os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune", "tuning.json"))


def _device_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load(cache):
    try:
        with open(cache) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(cache, key, entry):
    data = _load(cache)
    data[key] = entry
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tmp = cache + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, cache)


def cache_key(signature: str, device: str | None = None) -> str:
    return f"{device or _device_name()}|{signature}"


def cached(signature: str, cache: str = DEFAULT_CACHE, device: str | None = None):
    """The cached winner for this device and workload signature, or None."""
    return _load(cache).get(cache_key(signature, device))


def _time_steps(sim, steps):
    import torch
    stream = torch.cuda.ExternalStream(sim.stream) if sim.stream else torch.cuda.current_stream()
    sim.step_async(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step_async(steps)
    e1.record(stream)
    e1.synchronize()
    sim.sync()
    return e0.elapsed_time(e1) / steps


def _apply(sim, cand, knob, choices):
    """Apply cand; if the context refuses it, the same with one other knob back at its first
    choice (the first such combination it accepts).  Returns the applied tuning or None."""
    try:
        sim.set_tuning(**cand)
        return cand
    except GrpicError:
        pass
    for other, vals in choices.items():
        if other == knob or cand[other] == vals[0]:
            continue
        alt = dict(cand, **{other: vals[0]})
        try:
            sim.set_tuning(**alt)
            return alt
        except GrpicError:
            continue
    return None


def tune(sim, signature: str, steps: int = 4, rounds: int = 2, cache: str = DEFAULT_CACHE, choices=CHOICES,
         use_cache: bool = True, timer=_time_steps, device: str | None = None):
    """Tune `sim` (a grpic.Simulation) in place; returns {"tuning": {...}, "ms_per_step": t,
    "trials": n, "cached": bool}.  The winner is applied to `sim` and written to the cache.
    steps should be a multiple of every sort interval tried, so each trial sorts a whole number
    of times."""
    if use_cache:
        hit = cached(signature, cache, device)
        if hit is not None:
            sim.set_tuning(**hit["tuning"])
            return dict(hit, cached=True, trials=0)
    cur = sim.tuning()
    best_ms = None
    trials = 0
    for _ in range(rounds):
        changed = False
        for knob, values in choices.items():
            times, combos = {}, {}
            for v in list(values) + list(values)[::-1]:
                cand = _apply(sim, dict(cur, **{knob: v}), knob, choices)
                if cand is None:
                    continue
                combos[v] = cand
                times.setdefault(v, []).append(timer(sim, steps))
                trials += 1
            results = {v: sum(t) / len(t) for v, t in times.items()}
            v_best = min(results, key=results.get)
            if combos[v_best] != cur:
                changed = True
            cur = combos[v_best]
            best_ms = results[v_best]
        if not changed:
            break
    sim.set_tuning(**cur)
    entry = {"tuning": cur, "ms_per_step": best_ms}
    _store(cache, cache_key(signature, device), entry)
    return dict(entry, cached=False, trials=trials)


def tune_batch(batch_step, set_blocks, signature: str, steps: int = 3, cache: str = DEFAULT_CACHE,
               choices=BATCH_CHOICES, use_cache: bool = True, device: str | None = None):
    """Tune the persistent blocks per SM of a batched engine.  batch_step(n) runs n synchronised
    batched steps and returns their wall time in ms; set_blocks(b) applies a choice."""
    if use_cache:
        hit = cached(signature, cache, device)
        if hit is not None:
            set_blocks(hit["tuning"]["batch_blocks_per_sm"])
            return dict(hit, cached=True, trials=0)
    results = {}
    for b in choices:
        set_blocks(b)
        batch_step(1)
        results[b] = batch_step(steps) / steps
    b_best = min(results, key=results.get)
    set_blocks(b_best)
    entry = {"tuning": {"batch_blocks_per_sm": b_best}, "ms_per_step": results[b_best]}
    _store(cache, cache_key(signature, device), entry)
    return dict(entry, cached=False, trials=len(choices))
