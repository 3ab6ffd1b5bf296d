#!/usr/bin/env python
"""Throughput of the GRPIC timestep on GB300.

Workload (one GPU): Kerr a = 0.9 m, m = 4 cells, 128^3 grid, electron-ion plasma (mass ratio
20), 8 particles per cell per species, u_th = 0.05 c, uniform contravariant B_z = 0.1,
dt = 0.4 -- synthetic, seeded (paper_0904_0232_gb300.synth.kerr_ion_electron_128).

A step is one whole cycle of the method: B half-step, push + deposit, B half-step, E step,
removal + counting sort.  ``value`` counts particle-steps per second in the FP32-mixed path
with inputs resident in HBM; the FP64 path is measured on the same state for comparison;
``e2e`` repeats the measurement through the C ABI with host buffers (load, steps, read back).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl grpic|reference]

N > 1 (torchrun) runs N independent replicas, one per GPU (weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+RK4 Kerr push+deposit) FP32-mixed vs FP64; p50/p99 latency"
UNIT = "particle-steps/s"

# Arithmetic operations per particle-step of the push + deposit, by Gauss-Legendre order Q of
# Eq. 18: the count of a plain restatement of the method's particle-step on a counting scalar
# (add, subtract, multiply, divide, square root = 1; FMA = 2), whose particle-step equals the
# oracle's to rounding -- tests/golden/flop_count.json, checked by tests/test_flop_count.py.  The
# kernels reach the same result with fewer operations; the numerator stays this count.
ALG_FLOPS = {1: 3401, 2: 6641, 3: 12041}

# Nominal FP32 CUDA-core peak of GB300: 152 SMs x 128 lanes x 2 flops x 2070 MHz.
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.070e9

# DRAM bytes per particle-step of the per-warp select push kernel (dram__bytes_read +
# dram__bytes_write of one launch over its particles), from ncu captures at the bench size, per
# variant (far-field area fits on or off, resident blocks per SM), valid for the push sources whose
# hash is recorded with them.
PUSH_TRAFFIC = {"sha": "6af44e8d10042355",
                "bytes_per_particle": {"area_table0_minb4": 1371.6e6 / 15.61e6,
                                       "area_table0_minb5": 1376.4e6 / 15.61e6,
                                       "area_table1_minb5": 2073.7e6 / 15.61e6}}


def push_variant(tuning):
    """Key of PUSH_TRAFFIC for a tuning dict (None: the per-warp push with its default shapes)."""
    t = tuning or {}
    if t.get("split", 0) != 0:
        return None
    return f"area_table{int(t.get('area_table', 0))}_minb{int(t.get('far_min_blocks', 4))}"


def kernel_sha():
    h = hashlib.sha256()
    for f in ("push.cu", "push_far.cu", "push_core.cuh", "metric.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_0904_0232_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["grpic", "reference"], default="grpic")
    p.add_argument("--grid", type=int, default=128)
    p.add_argument("--quad", type=int, default=2)
    p.add_argument("--sort-interval", type=int, default=1)
    p.add_argument("--fp64-steps", type=int, default=20,
                   help="steps of the FP64 comparison leg (at most --steps), after the same warm-up as the "
                        "measured window; 0 skips it")
    p.add_argument("--fp64-late-steps", type=int, default=10,
                   help="steps of the FP64 and FP32-mixed legs from the state at the end of the measured "
                        "window (read back by the end-to-end leg); 0 skips them")
    p.add_argument("--fp32-compare-steps", type=int, default=200,
                   help="steps of the all-FP32 comparison run (no FP64 region); 0 skips it")
    p.add_argument("--workload", choices=["kerr128", "batch", "disk384", "jet", "fields"], default="kerr128",
                   help="kerr128: the single-instance Kerr electron-ion workload; batch: many small "
                        "instances advanced by the batched engine; disk384: the 384^3 disk/corona plasma "
                        "(~1e9 particles, generated on the device); jet: the parameters of the paper's "
                        "application set-up (64x64x128, c = 0.05, ~0.97 million particles); fields: the field "
                        "stages alone (B half-steps, E step) on an n^3 Kerr grid without particles")
    p.add_argument("--single-kernel-steps", type=int, default=200,
                   help="steps of the comparison run with the single mixed push kernel; 0 skips it")
    p.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no autotuning)")
    p.add_argument("--tuning", default=None,
                   help="launch shapes as a JSON object of grpic_tuning fields (no autotuning), e.g. "
                        "'{\"far_min_blocks\": 5, \"spread\": 16, \"sort_interval\": 4}'")
    p.add_argument("--batch-n", type=int, default=64)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


# ---- distributed plumbing (replicas) ---------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as td

            td.init_process_group("gloo")
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        if not self.pg:
            return v
        import torch

        t = torch.tensor([float(v)], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v):
        if not self.pg:
            return v
        import torch

        t = torch.tensor([float(v)], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---- clocks sampled during the timed region ---------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU baseline (the oracle, as it stands) ---------------------------------------------------
def cpu_sample_workload():
    """Bounded CPU sample: the Kerr electron-ion workload's parameters on a 40^3 window around
    the hole, 20,000 evenly strided particles per species."""
    from paper_0904_0232_gb300 import synth

    return synth.subsample(synth.kerr_ion_electron_128(seed=2, n=40), 20000)


def run_oracle_steps(wl, steps, warmup=0, threads=0):
    import oracle as O

    o = O.Oracle(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, threads=threads)
    o.init_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        o.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=1)
    for _ in range(warmup):
        o.step(1)
    n_before = sum(o.num_particles(s) for s in range(len(wl.species)))
    t0 = time.perf_counter()
    psteps = 0
    per_step = []
    for _ in range(steps):
        n = sum(o.num_particles(s) for s in range(len(wl.species)))
        t1 = time.perf_counter()
        o.step(1)
        per_step.append(time.perf_counter() - t1)
        psteps += n
    el = time.perf_counter() - t0
    del n_before
    return psteps, el, (threads if threads > 0 else O.max_threads()), per_step


def cpu_baseline(steps=150, single_thread_steps=5):
    """The oracle on all host cores over `steps` steps of the sample, and on one thread over its
    first `single_thread_steps` steps."""
    wl = cpu_sample_workload()
    psteps, el, cores, _ = run_oracle_steps(wl, steps)
    out = {"value": psteps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"FP64 oracle, Kerr a=0.9m m=4 on a {wl.nx}^3 window, {wl.n_particles} particles "
                     f"(2 species), {steps} whole steps incl. field solve; {el:.1f} s wall"}
    if single_thread_steps > 0:
        ps1, el1, _, _ = run_oracle_steps(wl, single_thread_steps, threads=1)
        out["single_thread"] = {"value": ps1 / el1, "unit": UNIT, "cores": 1,
                                "sample": f"the first {single_thread_steps} steps of the same sample; {el1:.1f} s wall"}
    return out


def run_reference(args, dist):
    if dist.rank != 0:
        return None
    wl = cpu_sample_workload()
    psteps, el, cores, per = run_oracle_steps(wl, args.steps, warmup=args.warmup)
    v = psteps / el
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "kerr_ion_electron_128 (bounded CPU sample: 40^3 window around the hole, "
                                   "40000 strided particles)",
                       "grid": wl.nx, "particles": wl.n_particles, "m": wl.m, "a": wl.a, "dt": wl.dt},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle steps of the 40^3 / 40000-particle sample"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---- GPU arm ------------------------------------------------------------------------------------
def pinned_empty(shape, dtype):
    """A numpy array over page-locked host memory (torch's pinned allocator)."""
    import torch

    tdt = {np.dtype(np.float64): torch.float64, np.dtype(np.int32): torch.int32}[np.dtype(dtype)]
    return torch.empty(shape, dtype=tdt, pin_memory=True).numpy()


def pinned_copy(a):
    out = pinned_empty(a.shape, a.dtype)
    out[...] = a
    return out


def make_sim(wl, precision, args, device_inputs=True, fp64_radius=0.0, flags=0, tuning=None):
    import torch

    from paper_0904_0232_gb300.grpic import GRPIC_U_COV_SPATIAL, Simulation

    sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision=precision, quad_order=args.quad,
                     sort_interval=args.sort_interval, fp64_radius=fp64_radius, flags=flags)
    if tuning is not None:
        sim.set_tuning(**tuning)
    sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        if device_inputs:
            x = torch.from_numpy(sp.x4).cuda()
            u = torch.from_numpy(np.vstack([sp.usp, np.zeros((1, sp.usp.shape[1]))])).cuda()
            i = torch.from_numpy(sp.ids.view(np.int32)).cuda()
            sim.load_particles(s, sp.q_over_m, sp.q_macro, x, u, i, umode=GRPIC_U_COV_SPATIAL)
            del x, u, i
        else:
            sim.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=GRPIC_U_COV_SPATIAL)
    torch.cuda.synchronize()
    return sim


def timed_steps(sim, steps, dist):
    import torch

    stream = torch.cuda.current_stream()
    sim.sync()
    st0 = sim.stats()["particle_steps"]
    sim.profile(reset=True)
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step_async(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms = e0.elapsed_time(e1)
    sim.sync()
    prof, launches = sim.profile(reset=True)
    psteps = sim.stats()["particle_steps"] - st0
    return ms, psteps, prof, launches


def run_gpu(args, dist):
    import torch

    from paper_0904_0232_gb300 import synth
    from paper_0904_0232_gb300.build import build
    from paper_0904_0232_gb300 import autotune
    from paper_0904_0232_gb300.grpic import GRPIC_FP32_MIXED, GRPIC_SINGLE_PUSH_KERNEL, grpic_probe_fma_peak

    torch.cuda.set_device(dist.local)
    build()
    wl = synth.kerr_ion_electron_128(seed=2, n=args.grid)

    # --- launch shapes from the autotuner, on a context of its own (tuning advances its state)
    sig = f"kerr_ion_electron_{args.grid}|Q{args.quad}|{wl.n_particles}"
    if args.tuning:
        tuned = {"tuning": json.loads(args.tuning), "cached": False, "trials": 0, "ms_per_step": None}
    elif args.no_tune:
        tuned = {"tuning": None, "cached": False, "trials": 0, "ms_per_step": None}
    else:
        simt = make_sim(wl, "fp32_mixed", args)
        tuned = autotune.tune(simt, sig, steps=8)
        simt.close()
        del simt
        torch.cuda.empty_cache()

    invariants = {}

    def leg(precision, steps, warmup, record_invariants=False, **kw):
        """A fresh context from the same initial state, `warmup` untimed then `steps` timed steps
        (with record_invariants, the invariant statistics over the timed steps, evaluated outside
        the timed region)."""
        s_ = make_sim(wl, precision, args, tuning=tuned["tuning"], **kw)
        s_.set_profiling(True)
        s_.step(warmup)
        if record_invariants:
            invariants["start"] = s_.invariants(baseline=True)
        out = timed_steps(s_, steps, dist) + (s_.stats(), s_.tuning())
        if record_invariants:
            invariants["end"] = s_.invariants()
        s_.close()
        del s_
        torch.cuda.empty_cache()
        return out

    def summary(ms_, ps_, prof_, steps, note=None):
        d = {"value": dist.sum(ps_) / (dist.max(ms_) * 1e-3), "unit": UNIT, "steps": steps,
             "ms_per_step": ms_ / steps, "push_ms_per_step": prof_["push_deposit"][0] / steps}
        if note:
            d["note"] = note
        return d

    # --- FP32-mixed, inputs resident in HBM
    clocks = Clocks(dist.local)
    clocks.start()
    ms, psteps, prof, launches, st, tuning_used = leg("fp32_mixed", args.steps, args.warmup, record_invariants=True)
    clk = clocks.stop()

    t_max = dist.max(ms)
    psteps_all = dist.sum(psteps)
    value = psteps_all / (t_max * 1e-3)

    push_ms, push_n = prof["push_deposit"]
    flops = ALG_FLOPS[args.quad] * psteps
    achieved = flops / (push_ms * 1e-3) if push_ms > 0 else 0.0
    fp32_probe = grpic_probe_fma_peak(GRPIC_FP32_MIXED)
    sha = kernel_sha()
    traffic = None
    per_particle = PUSH_TRAFFIC["bytes_per_particle"].get(push_variant(tuning_used))
    if PUSH_TRAFFIC["sha"] == sha and per_particle:
        traffic = per_particle * psteps / max(1, push_n)

    # --- end to end through the C ABI with host buffers: the inputs and outputs live in pinned host
    # memory (prepared before the timed region, as a caller's staging buffers would be); inside it:
    # context creation, field init, particle load (host -> device, u^4 completed), K steps, and the
    # read-back of every particle and field.  It runs right after the main leg, in the process state a
    # user's program has: after the comparison legs below, the read-back's staging allocations were
    # 3-8x slower (the caching allocator's state), which is not the library's cost.
    e2e = None
    late = None
    if not args.no_e2e:
        import ctypes

        from paper_0904_0232_gb300.grpic import (GRPIC_MEM_HOST, GRPIC_U_COV_SPATIAL, Simulation, grpic_num_particles,
                                                 load_library)

        host_in, host_out = [], []
        for sp in wl.species:
            n = sp.x4.shape[1]
            u = np.vstack([sp.usp, np.zeros((1, n))])
            host_in.append((pinned_copy(sp.x4), pinned_copy(u), pinned_copy(sp.ids.view(np.int32)).view(np.uint32)))
            host_out.append((pinned_empty((4, n), np.float64), pinned_empty((4, n), np.float64),
                             pinned_empty((n,), np.int32).view(np.uint32)))
        fshape = (3, wl.nz, wl.ny, wl.nx)
        fields_out = [pinned_empty(fshape, np.float64) for _ in range(3)]
        d_h2d = sum(x.nbytes + u.nbytes + i.nbytes for x, u, i in host_in)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        lib = load_library()
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision="fp32_mixed", quad_order=args.quad,
                         sort_interval=args.sort_interval)
        if tuned["tuning"] is not None:
            sim.set_tuning(**tuned["tuning"])
        t1 = time.perf_counter()
        sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
        for s, (sp, (x, u, i)) in enumerate(zip(wl.species, host_in)):
            sim.load_particles(s, sp.q_over_m, sp.q_macro, x, u, i, umode=GRPIC_U_COV_SPATIAL)
        sim.sync()
        t2 = time.perf_counter()
        sim.step_async(args.steps)
        sim.sync()
        t3 = time.perf_counter()
        out_bytes = 0
        counts = []
        for s, (x, u, i) in enumerate(host_out):
            nn = ctypes.c_int64(x.shape[1])
            assert lib.grpic_get_particles(sim.handle, s, ctypes.byref(nn), ptr(x), ptr(u), ptr(i), GRPIC_MEM_HOST) == 0
            out_bytes += nn.value * (x.itemsize * 8 + i.itemsize)
            counts.append(nn.value)
        assert lib.grpic_get_fields(sim.handle, *(ptr(f) for f in fields_out), GRPIC_MEM_HOST) == 0
        out_bytes += sum(f.nbytes for f in fields_out)
        torch.cuda.synchronize()
        el = el_local = time.perf_counter() - t0
        ps_e2e = sim.stats()["particle_steps"]
        sim.close()
        el = dist.max(el)
        e2e = {"value": dist.sum(ps_e2e) / el, "unit": UNIT, "h2d_bytes_per_step": int(d_h2d / args.steps),
               "d2h_bytes_per_step": int(out_bytes / args.steps),
               "phases_ms": {"create_and_tune": round((t1 - t0) * 1e3, 1), "fields_and_load": round((t2 - t1) * 1e3, 1),
                             "steps": round((t3 - t2) * 1e3, 1), "readback": round((t0 + el_local - t3) * 1e3, 1)},
               "includes": "context creation, field init, particle load from pinned host memory (u^4 completed on "
                           "the device), K steps, read-back of every particle and field into pinned host memory"}
        if args.fp64_late_steps > 0:
            late = late_window(wl, args, dist, tuned["tuning"], host_out, counts, fields_out, summary)
        del host_in, host_out, fields_out

    # --- the FP64 path over the measured window (its first steps when --steps is longer; it runs at a
    #     small fraction of the FP32 rate), beside the FP32-mixed path over the same steps
    fp64 = None
    n64 = min(args.fp64_steps, args.steps)
    if n64 > 0:
        ms64, ps64, prof64, _, _, _ = leg("fp64", n64, args.warmup)
        if n64 == args.steps:
            msw, psw, profw = ms, psteps, prof
        else:
            msw, psw, profw, _, _, _ = leg("fp32_mixed", n64, args.warmup)
        fp64 = summary(ms64, ps64, prof64, n64, f"steps {args.warmup + 1}-{args.warmup + n64} from the start")
        fp64["fp32_mixed_same_window"] = summary(msw, psw, profw, n64)
        if profw["push_deposit"][0] > 0:
            # the push's fraction over these early steps, before particles gather near the hole
            early_frac = ALG_FLOPS[args.quad] * psw / (profw["push_deposit"][0] * 1e-3) / FP32_PEAK_NOMINAL
            fp64["fp32_mixed_same_window"]["push_roofline_frac"] = early_frac

    # --- the same steps with every particle through the FP32-mixed code (no far-field path)
    single = None
    if args.single_kernel_steps > 0:
        ms1, ps1, prof1, _, _, _ = leg("fp32_mixed", args.single_kernel_steps, args.warmup,
                                       flags=GRPIC_SINGLE_PUSH_KERNEL)
        single = summary(ms1, ps1, prof1, args.single_kernel_steps,
                         "GRPIC_SINGLE_PUSH_KERNEL: every particle through the FP32-mixed code")

    # --- the same steps with the FP64 region switched off (all-FP32 metric evaluations)
    fp32_all = None
    if args.fp32_compare_steps > 0:
        ms32, ps32, prof32, _, _, _ = leg("fp32_mixed", args.fp32_compare_steps, args.warmup, fp64_radius=-1.0)
        fp32_all = summary(ms32, ps32, prof32, args.fp32_compare_steps,
                           "fp64_radius < 0: no FP64 metric evaluations (the FP32-only comparison; its particle error against "
                           "the FP64 oracle after one push is ~1e-7 relative, like the policy's)")

    cpu = None
    if dist.rank == 0 and not args.no_cpu:
        cpu = cpu_baseline()

    stage_ms = {k: round(v[0] / max(1, args.steps), 4) for k, v in prof.items()}
    hbm_stages = hbm_stage_summary(prof, args.steps, wl.nx * wl.ny * wl.nz, psteps / max(1, args.steps),
                                   tuning_used.get("sort_interval", args.sort_interval))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64 quartic/metric/Christoffel where r < 4m; FP64 J)",
        "data": "synthetic (seeded generator; stands in for the paper's disk/corona plasma)",
        "config": {"workload": f"kerr_ion_electron_{args.grid}: Kerr a=0.9m, m=4 cells, {args.grid}^3 grid, "
                               "e-/ion (mass ratio 20), 8 ppc per species, u_th=0.05c, B_z=0.1, dt=0.4",
                   "particles": wl.n_particles, "quad_order": args.quad,
                   "tuning": dict(tuning_used, autotuned=not (args.no_tune or args.tuning), cached=tuned["cached"],
                                  trials=tuned["trials"]),
                   "window": f"steps {args.warmup + 1}-{args.warmup + args.steps} from the start; every "
                             "comparison leg starts from the same state",
                   "parallelism": f"replicas x{dist.world}",
                   "l2": "inputs larger than L2 (particle store %.2f GB)" % (wl.n_particles * 40 / 1e9)},
        "gpu_launches": int(launches),
        "stage_ms_per_step": stage_ms,
        "hbm_stages": hbm_stages,
        "roofline": {"kernel": "push stage (k_push_select: far-field FP32 or FP32-mixed code per warp; with "
                               "tuning split=1 the k_classify_near + k_push_near + k_push_far kernels)",
                     "bound": "alu", "achieved": achieved / 1e12,
                     "peak": FP32_PEAK_NOMINAL / 1e12, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_NOMINAL,
                     "traffic": traffic, "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal)",
                     "fma_probe_tflops": fp32_probe / 1e12,
                     "flops_per_particle_step": ALG_FLOPS[args.quad], "kernel_sha": sha},
        "fp64": fp64,
        "fp64_late_window": late,
        "single_push_kernel": single,
        "fp32_no_fp64_region": fp32_all,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
        "stats": {k: st[k] for k in ("removed_horizon", "removed_outer", "gamma_fallbacks", "fp64_evals")},
        "invariants": invariant_summary(invariants["start"], invariants["end"], args.steps),
    }
    return line


def planar_head(buf, n):
    """The (4, n) planar array grpic_get_particles wrote into the front of buf: its planes are n
    (the count written) apart, not buf's row length (the capacity)."""
    return buf.reshape(-1)[:4 * n].reshape(4, n)


def late_window(wl, args, dist, tuning, host_out, counts, fields_out, summary):
    """The FP64 path against the FP32-mixed path at the END of the measured window, where the most
    particles have gathered near the hole: both start from the state the end-to-end leg read back
    after its K steps (every particle with its full u^a and own clock, and the fields b, d), take
    one untimed step, then --fp64-late-steps timed steps."""
    import torch

    from paper_0904_0232_gb300.grpic import GRPIC_U_FULL, Simulation

    out = {}
    try:
        for precision in ("fp64", "fp32_mixed"):
            s_ = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision=precision, quad_order=args.quad,
                            sort_interval=args.sort_interval)
            if tuning is not None:
                s_.set_tuning(**tuning)
            s_.set_fields(fields_out[0], fields_out[1])
            for sidx, (sp, (x, u, i), nn) in enumerate(zip(wl.species, host_out, counts)):
                s_.load_particles(sidx, sp.q_over_m, sp.q_macro, planar_head(x, nn), planar_head(u, nn), i[:nn],
                                  umode=GRPIC_U_FULL)
            s_.set_profiling(True)
            s_.step(1)
            ms_, ps_, prof_, _ = timed_steps(s_, args.fp64_late_steps, dist)
            s_.close()
            del s_
            torch.cuda.empty_cache()
            out[precision] = summary(ms_, ps_, prof_, args.fp64_late_steps)
    except Exception as exc:  # a comparison leg: report, do not lose the line
        return {"error": repr(exc)}
    k = args.fp64_late_steps
    out["note"] = (f"steps {args.steps + 2}-{args.steps + 1 + k} of a run (from the state after the end-to-end leg's "
                   f"{args.steps} steps, one untimed step)")
    return out


def invariant_summary(start, end, steps):
    """Per-run invariant statistics: the normalisation residual |g(u,u) + c^2| / c^2 (Eq. 7) at the
    start and the end of the timed steps, and the change of E = -u_4 and L = u_phi (Eq. 3) over them
    for the tracked subsample (ids divisible by 64) -- E and L are invariants of field-free orbits
    only; with fields they measure the work done on the particles."""
    return {"steps": steps, "norm_max_start": start["norm_max"], "norm_max": end["norm_max"],
            "norm_mean": end["norm_mean"], "tracked": end["tracked"],
            "energy_change_mean": end["energy_mean"], "energy_change_max": end["energy_max"],
            "angmom_change_mean": end["angmom_mean"], "angmom_change_max": end["angmom_max"],
            "units": "norm relative to c^2; E and L changes divided by c (L in cells)"}


def run_batch(args, dist):
    """Batched workload: n instances (grids 32^3-96^3, 1-32 particles per cell per species,
    m in [1, 4] cells, a in [0, 0.99] m, pair plasma, B_z = 0.05, dt = 0.4, FP32-mixed) advanced
    by one persistent launch per stage from a CUDA graph; compared with the same instances
    stepped one after another."""
    import torch

    from paper_0904_0232_gb300 import synth
    from paper_0904_0232_gb300.build import build
    from paper_0904_0232_gb300 import autotune
    from paper_0904_0232_gb300.grpic import (GRPIC_U_COV_SPATIAL, Simulation, grpic_batch_create,
                                             grpic_batch_destroy, grpic_batch_info, grpic_batch_set_blocks_per_sm,
                                             grpic_batch_step)

    torch.cuda.set_device(dist.local)
    build()
    specs = synth.batch_specs(args.batch_n)
    dev = torch.device("cuda")
    draws = {}
    for g in sorted({sp.grid for sp in specs}):
        x, u0, u1 = synth.cell_major_pairs(g, 32, 0.1, 1.0, seed=7)
        draws[g] = tuple(torch.from_numpy(a).to(dev) for a in (x, u0, u1))
    sims = []
    npart = 0
    for k, sp in enumerate(specs):
        x, u0, u1 = draws[sp.grid]
        xs = x[:, :, :sp.ppc].reshape(3, -1)
        n = xs.shape[1]
        x4 = torch.cat([xs, torch.zeros((1, n), dtype=torch.float64, device=dev)]).contiguous()
        ids = torch.arange(n, dtype=torch.int32, device=dev)
        q = synth.charge_for(0.4, sp.ppc, (-1.0, 1.0), 0.1)
        sim = Simulation(sp.grid, sp.grid, sp.grid, sp.m, sp.a, 1.0, 0.4, precision="fp32_mixed",
                         quad_order=args.quad)
        sim.set_uniform_field(B=(0.0, 0.0, 0.05))
        for s, (qm, u) in enumerate(((-1.0, u0), (1.0, u1))):
            us = torch.cat([u[:, :, :sp.ppc].reshape(3, -1), torch.zeros((1, n), dtype=torch.float64, device=dev)])
            sim.load_particles(s, qm, float(np.sign(qm) * q), x4, us.contiguous(), ids, umode=GRPIC_U_COV_SPATIAL)
        npart += sum(sim.num_particles(s) for s in range(2))
        sims.append(sim)
    del draws
    torch.cuda.empty_cache()

    def psteps():
        return sum(s.stats()["particle_steps"] for s in sims)

    b = grpic_batch_create([s.handle for s in sims])
    kps, blocks = grpic_batch_info(b)

    def run_steps(k):
        torch.cuda.synchronize()
        t = time.perf_counter()
        grpic_batch_step(b, k)
        return 1e3 * (time.perf_counter() - t)

    if args.no_tune:
        tuned = {"tuning": {"batch_blocks_per_sm": 8}, "cached": False, "trials": 0}
    else:
        tuned = autotune.tune_batch(run_steps, lambda v: grpic_batch_set_blocks_per_sm(b, v),
                                    f"batch{len(specs)}|Q{args.quad}|{npart}")
    grpic_batch_step(b, args.warmup)
    p0 = psteps()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grpic_batch_step(b, args.steps)
    el = time.perf_counter() - t0
    batched = (psteps() - p0) / el
    grpic_batch_destroy(b)
    # the same instances one after another (one context's step sequence at a time)
    seq_steps = max(1, min(args.steps, 10))
    p0 = psteps()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in sims:
        s.step_async(seq_steps)
    for s in sims:
        s.sync()
    el_seq = time.perf_counter() - t0
    sequential = (psteps() - p0) / el_seq
    value = dist.sum(batched)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 quartic/metric/Christoffel where r < 4m; FP64 J)",
            "data": "synthetic (seeded generator)",
            "config": {"workload": f"batch of {len(specs)} instances: grids 32^3-96^3, 1-32 ppc per species, "
                                   "m 1-4 cells, a 0-0.99 m, pair plasma, B_z=0.05, dt=0.4, omega_p dt=0.1",
                       "particles": npart, "kernels_per_step": kps, "work_blocks": blocks,
                       "tuning": dict(tuned["tuning"], autotuned=not args.no_tune, cached=tuned["cached"],
                                      trials=tuned["trials"]),
                       "timing": "host wall clock around synchronising graph replays"},
            "sequential": {"value": sequential, "unit": UNIT, "steps": seq_steps,
                           "note": "the same contexts stepped one after another (non-batched launches)"},
            "gpu_launches": int(kps * args.steps)}
    for s in sims:
        s.close()
    return line


def run_disk(args, dist):
    """The largest configuration: Kerr a = 0.95 m, m = 8, 384^3, accretion disk in a corona,
    ~1e9 particles generated on the device, FP32-mixed; particle-steps/s over K steps."""
    import torch

    from paper_0904_0232_gb300 import synth_disk
    from paper_0904_0232_gb300.build import build
    from paper_0904_0232_gb300.grpic import Simulation

    torch.cuda.set_device(dist.local)
    build()
    wl = synth_disk.kerr_disk_corona(n=args.grid if args.grid != 128 else 384, seed=3)
    npart = wl.n_particles
    layers = dict(wl.layers)
    sim = Simulation(wl.n, wl.n, wl.n, wl.m, wl.a, wl.c, wl.dt, precision="fp32_mixed", quad_order=args.quad,
                     **layers)
    tuning = json.loads(args.tuning) if args.tuning else {"sort_interval": args.sort_interval}
    sim.set_tuning(**tuning)
    sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
    for s, sp in enumerate(wl.species):
        sim.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.u4, sp.ids, umode=sp.umode)
    geo = dict(n=wl.n, m=wl.m, a=wl.a, n0=round(wl.n0, 1))
    del wl, sp
    torch.cuda.empty_cache()
    sim.set_profiling(True)
    sim.step(args.warmup)
    inv0 = sim.invariants(baseline=True)
    clocks = Clocks(dist.local)
    clocks.start()
    ms, psteps, prof, launches = timed_steps(sim, args.steps, dist)
    clk = clocks.stop()
    inv1 = sim.invariants()
    st = sim.stats()
    sim.close()
    value = dist.sum(psteps) / (dist.max(ms) * 1e-3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dist.max(ms) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 quartic/metric/Christoffel where r < 4m; FP64 J)",
            "invariants": invariant_summary(inv0, inv1, args.steps),
            "data": "synthetic (device-generated disk + corona)",
            "config": {"workload": f"kerr_disk_corona_{geo['n']}: Kerr a=0.95m, m={geo['m']:g} cells, {geo['n']}^3, "
                                   "Keplerian disk (|z|<0.1 r_cyl, 6m..150 cells, density ~1/r) in a 1% corona, "
                                   "e-/ion (mass ratio 20), B_z=0.1, dt=0.4",
                       "absorbing_layers": layers,
                       "particles": npart, "inner_edge_particles_per_cell": geo["n0"],
                       "tuning": tuning},
            "gpu_launches": int(launches),
            "stage_ms_per_step": {k: round(v[0] / max(1, args.steps), 4) for k, v in prof.items()},
            "clocks": clk,
            "stats": {k: st[k] for k in ("removed_horizon", "removed_outer", "gamma_fallbacks", "fp64_evals")}}


def run_jet(args, dist):
    """The application set-up of Sec. 6 (synth.kerr_jet_disk: 64 x 64 x 128, c = 0.05, dt = 1,
    a = 0.95 m, B_z = 30, |q/m| = 1e-3, 0.8 million disk particles in a free-falling corona),
    FP32-mixed, launch shapes from the autotuner; particle-steps/s over K steps."""
    import torch

    from paper_0904_0232_gb300 import autotune, synth
    from paper_0904_0232_gb300.build import build
    from paper_0904_0232_gb300.grpic import Simulation

    torch.cuda.set_device(dist.local)
    build()
    wl = synth.kerr_jet_disk(seed=4)

    def make(tuning=None):
        sim = Simulation(wl.nx, wl.ny, wl.nz, wl.m, wl.a, wl.c, wl.dt, precision="fp32_mixed", quad_order=args.quad,
                         sort_interval=args.sort_interval)
        if tuning is not None:
            sim.set_tuning(**tuning)
        sim.set_uniform_field(B=(0.0, 0.0, wl.B0))
        for s, sp in enumerate(wl.species):
            sim.load_particles(s, sp.q_over_m, sp.q_macro, sp.x4, sp.usp, sp.ids, umode=sp.umode)
        return sim

    tuning = None
    if not args.no_tune:
        simt = make()
        tuning = autotune.tune(simt, f"kerr_jet_disk_64x64x128|Q{args.quad}|{wl.n_particles}", steps=8)["tuning"]
        simt.close()
    sim = make(tuning)
    sim.set_profiling(True)
    sim.step(args.warmup)
    inv0 = sim.invariants(baseline=True)
    clocks = Clocks(dist.local)
    clocks.start()
    ms, psteps, prof, launches = timed_steps(sim, args.steps, dist)
    clk = clocks.stop()
    inv1 = sim.invariants()
    st = sim.stats()
    used = sim.tuning()
    sim.close()
    value = dist.sum(psteps) / (dist.max(ms) * 1e-3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dist.max(ms) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 quartic/metric/Christoffel where r < 4m; FP64 J)",
            "data": "synthetic (seeded; the parameters of the paper's application set-up, Sec. 6)",
            "invariants": invariant_summary(inv0, inv1, args.steps),
            "config": {"workload": "kerr_jet_disk_64x64x128: Kerr a=0.95m, m=2 cells, c=0.05, dt=1, B_z=30, "
                                   "e-/e+ |q/m|=1e-3, Keplerian disk (R>12 cells, |cos theta|<1/8, 0.8M particles) "
                                   "at 100x the density of a free-falling corona",
                       "particles": wl.n_particles, "tuning": used,
                       "l2": "working set below L2 (particle store 31 MB): a small-workload measurement"},
            "gpu_launches": int(launches),
            "stage_ms_per_step": {k: round(v[0] / max(1, args.steps), 4) for k, v in prof.items()},
            "clocks": clk,
            "stats": {k: st[k] for k in ("removed_horizon", "removed_outer", "gamma_fallbacks", "fp64_evals")}}


# Algorithmic bytes per cell of the field stages in FP32 (words of 4 B; J is FP64): first B half-step
# reads b, d and writes b^n (9 words); the second, time-centred, also reads b^{n-1/2} (12 words); the
# E step reads b, d, J and writes d (9 words + 24 B); J = 0 writes 24 B.
FIELD_BYTES = {"b_half": 36, "b_half2": 48, "e_step": 60, "zero_j": 24}


# Sort: the key of every particle read by the histogram, then each 40-byte record (x^1..3, the
# clock offset, u^1..4 in FP32, id) read and written by the scatter.
SORT_BYTES = 4 + 2 * 40


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh).get("hbm_gbs", 6800.0)), "measured"
    except (OSError, ValueError):
        return 6800.0, "fallback"


def hbm_stage_summary(prof, steps, cells, particles, sort_interval):
    """The HBM-bound stages of a measured run (the field stages and the sort) against their
    algorithmic bytes: device time per step from the run's CUDA events, bytes per cell (fields) or
    per particle and sort (sort; one sort every sort_interval steps)."""
    hbm, src = measured_hbm_gbs()
    out = {"peak_gbs": hbm, "peak_source": src}
    for k, nbytes in FIELD_BYTES.items():
        if k not in prof or prof[k][0] <= 0:
            continue
        t = prof[k][0] / max(1, steps) * 1e-3
        gbs = nbytes * cells / t / 1e9
        out[k] = {"ms": round(t * 1e3, 4), "algorithmic_bytes": nbytes * cells, "gbs": round(gbs, 1),
                  "frac": round(gbs / hbm, 3)}
    if "sort" in prof and prof["sort"][0] > 0:
        t = prof["sort"][0] / max(1, steps) * 1e-3
        nbytes = SORT_BYTES * particles / max(1, sort_interval)
        gbs = nbytes / t / 1e9
        out["sort"] = {"ms": round(t * 1e3, 4), "algorithmic_bytes": nbytes, "gbs": round(gbs, 1),
                       "frac": round(gbs / hbm, 3), "sort_interval": sort_interval}
    return out


def run_fields(args, dist):
    """The field stages alone: Kerr a = 0.9 m, m = 4 cells (m = 8, a = 0.95 m and the disk
    workload's absorbing layers at n >= 256, the 384^3 disk geometry), n^3 grid, uniform B_z = 0.1,
    no particles, FP32-mixed; device time per stage from CUDA events over K whole cycles, against
    the stage's algorithmic bytes (those of the cells outside the layers)."""
    import torch

    from paper_0904_0232_gb300.build import build
    from paper_0904_0232_gb300.grpic import Simulation
    from paper_0904_0232_gb300.synth_disk import DiskCorona

    torch.cuda.set_device(dist.local)
    build()
    n = args.grid
    m, a = (8.0, 0.95 * 8.0) if n >= 256 else (4.0, 0.9 * 4.0)
    layers = DiskCorona("", n, m, a, 1.0, 0.4, 0.1, 0, 0.0, []).layers if n >= 256 else {}
    sim = Simulation(n, n, n, m, a, 1.0, 0.4, precision="fp32_mixed", **layers)
    sim.set_uniform_field(B=(0.0, 0.0, 0.1))
    sim.set_profiling(True)
    sim.step(args.warmup)
    clocks = Clocks(dist.local)
    clocks.start()
    ms, _, prof, launches = timed_steps(sim, args.steps, dist)
    clk = clocks.stop()
    sim.close()
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    cells = float(n) ** 3
    stages = {}
    for k, nbytes in FIELD_BYTES.items():
        t = prof[k][0] / max(1, args.steps) * 1e-3
        gbs = nbytes * cells / t / 1e9 if t > 0 else None
        stages[k] = {"ms": round(t * 1e3, 4), "algorithmic_bytes_per_cell": nbytes,
                     "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / hbm if gbs else None}
    return {"metric": "field stage time (B half-steps, E step)", "value": dist.max(ms) / args.steps, "unit": "ms/step",
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dist.max(ms) / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (uniform field, no particles)",
            "config": {"workload": f"fields_{n}: Kerr a={a / m:g}m, m={m:g} cells, {n}^3, B_z=0.1, dt=0.4, no particles",
                       "absorbing_layers": layers, "hbm_peak_gbs": hbm, "l2": "field planes larger than L2" if 15 * 4 * cells > 129e6
                       else "field planes fit in L2 (a small-grid measurement)"},
            "gpu_launches": int(launches), "stages": stages, "clocks": clk}


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        line = run_reference(args, dist)
    elif args.workload == "batch":
        line = run_batch(args, dist)
    elif args.workload == "disk384":
        line = run_disk(args, dist)
    elif args.workload == "jet":
        line = run_jet(args, dist)
    elif args.workload == "fields":
        line = run_fields(args, dist)
    else:
        line = run_gpu(args, dist)
    if dist.rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    dist.close()


if __name__ == "__main__":
    main()
