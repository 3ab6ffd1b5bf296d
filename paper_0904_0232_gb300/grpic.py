"""ctypes binding of the GRPIC C ABI (include/grpic.h): the same entry points under the same
names, plus a small ``Simulation`` convenience wrapper.  Argument marshalling only -- every
step of the timestep runs in the CUDA library.  Device memory comes from PyTorch's caching
allocator through the ABI's allocator callbacks, and work runs on PyTorch's current stream.

The library must be built first (``paper_0904_0232_gb300.build.build()``); loading fails
loudly if it is missing.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrpic.so")

GRPIC_OK = 0
STATUS_NAMES = {0: "GRPIC_OK", 1: "GRPIC_ERR_INVALID", 2: "GRPIC_ERR_OOM", 3: "GRPIC_ERR_CUDA", 4: "GRPIC_ERR_CFL",
                5: "GRPIC_ERR_NONFINITE", 6: "GRPIC_ERR_TIMEOUT", 7: "GRPIC_ERR_AGAIN", 8: "GRPIC_ERR_CAPACITY",
                9: "GRPIC_ERR_UNSTABLE"}
GRPIC_ERR_UNSTABLE = 9
GRPIC_FP64, GRPIC_FP32_MIXED = 0, 1
GRPIC_NO_GAMMA_IN_J = 1
GRPIC_LITERAL_HALF_STEPS = 2
GRPIC_SINGLE_PUSH_KERNEL = 4
GRPIC_MEM_HOST, GRPIC_MEM_DEVICE = 0, 1
GRPIC_U_FULL, GRPIC_U_COV_SPATIAL, GRPIC_U_CONTRA_SPATIAL, GRPIC_LOAD_DEVICE = 0, 1, 2, 16
GRPIC_STAGE_B_HALF, GRPIC_STAGE_ZERO_J, GRPIC_STAGE_PUSH_DEPOSIT, GRPIC_STAGE_E, GRPIC_STAGE_SORT, GRPIC_STAGE_B_HALF2 = range(6)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class grpic_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("m", ctypes.c_double), ("a", ctypes.c_double), ("c", ctypes.c_double), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int), ("quad_order", ctypes.c_int), ("r_excise", ctypes.c_double),
                ("flags", ctypes.c_uint), ("sort_interval", ctypes.c_int), ("max_particles", ctypes.c_int64),
                ("fp64_radius", ctypes.c_double), ("absorb_inner", ctypes.c_double),
                ("absorb_outer", ctypes.c_double), ("absorb_width", ctypes.c_int),
                ("z_origin", ctypes.c_int), ("nz_total", ctypes.c_int),
                ("alloc", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_user", ctypes.c_void_p)]


class grpic_request(ctypes.Structure):
    _fields_ = [("cfg", grpic_config), ("E_contra", ctypes.c_double * 3), ("B_contra", ctypes.c_double * 3),
                ("nspecies", ctypes.c_int), ("q_over_m", ctypes.c_double * 4), ("q_macro", ctypes.c_double * 4),
                ("ppc", ctypes.c_int), ("u_th", ctypes.c_double), ("r_min", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("nsteps", ctypes.c_int)]


GRPIC_RUN_QUEUED, GRPIC_RUN_RUNNING, GRPIC_RUN_DONE = 0, 1, 2


class grpic_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("removed_horizon", ctypes.c_int64), ("removed_outer", ctypes.c_int64),
                ("gamma_fallbacks", ctypes.c_int64), ("fp64_evals", ctypes.c_int64),
                ("particle_steps", ctypes.c_int64), ("n_alive", ctypes.c_int64 * 4)]


class grpic_invariants(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("norm_max", ctypes.c_double), ("norm_mean", ctypes.c_double),
                ("tracked", ctypes.c_int64), ("energy_mean", ctypes.c_double), ("energy_max", ctypes.c_double),
                ("angmom_mean", ctypes.c_double), ("angmom_max", ctypes.c_double)]


class grpic_tuning(ctypes.Structure):
    _fields_ = [("far_min_blocks", ctypes.c_int), ("near_blocks_per_sm", ctypes.c_int), ("sort_interval", ctypes.c_int),
                ("overlap", ctypes.c_int), ("split", ctypes.c_int), ("j_tile", ctypes.c_int),
                ("spread", ctypes.c_int), ("area_table", ctypes.c_int)]


EXPORTS = {
    "grpic_create": (ctypes.c_int, [ctypes.POINTER(grpic_config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "grpic_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "grpic_set_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "grpic_set_uniform_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]),
    "grpic_set_j": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "grpic_get_fields_contra": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "grpic_get_planes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int]),
    "grpic_set_planes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_int]),
    "grpic_load_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int]),
    "grpic_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grpic_step_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grpic_stage": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grpic_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "grpic_get_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int]),
    "grpic_num_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "grpic_get_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "grpic_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(grpic_stats)]),
    "grpic_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "grpic_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "grpic_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grpic_get_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                         ctypes.c_int]),
    "grpic_get_invariants": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(grpic_invariants)]),
    "grpic_charge_density": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "grpic_gauss_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_double)]),
    "grpic_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(grpic_tuning)]),
    "grpic_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(grpic_tuning)]),
    "grpic_probe_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "grpic_check_newton64": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    "grpic_check_conversions": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "grpic_sort_particles_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p]),
    "grpic_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ALLOC_FN, FREE_FN, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "grpic_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(grpic_request), ctypes.POINTER(ctypes.c_uint64)]),
    "grpic_server_tick": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "grpic_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "grpic_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "grpic_request_bytes": (ctypes.c_int, [ctypes.POINTER(grpic_request), ctypes.POINTER(ctypes.c_size_t)]),
    "grpic_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "grpic_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "grpic_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grpic_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "grpic_batch_set_blocks_per_sm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "grpic_batch_ctx_status": (ctypes.c_int, [ctypes.c_void_p]),
    "grpic_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgrpic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_0904_0232_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GrpicError(RuntimeError):
    def __init__(self, code, where, msg=""):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} {msg}".strip())
        self.code = code


# ---- PyTorch-backed device allocator --------------------------------------------------------
def _torch():
    import torch

    return torch


@ALLOC_FN
def _torch_alloc(nbytes, user):
    torch = _torch()
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  torch.cuda.current_stream())
    except Exception:  # out of memory -> NULL -> GRPIC_ERR_OOM
        return None


@FREE_FN
def _torch_free(ptr, user):
    if ptr and sys.meta_path is not None:  # at interpreter shutdown the process frees everything
        _torch().cuda.caching_allocator_delete(ptr)


# ---- thin wrappers with the ABI's names ------------------------------------------------------
def _check(ctx, code, where):
    if code != GRPIC_OK:
        msg = load_library().grpic_last_error(ctx).decode() if ctx else ""
        raise GrpicError(code, where, msg)


def grpic_create(cfg: grpic_config, stream=None):
    h = ctypes.c_void_p()
    code = load_library().grpic_create(ctypes.byref(cfg), stream, ctypes.byref(h))
    if code != GRPIC_OK:
        raise GrpicError(code, "grpic_create")
    return h.value


def grpic_destroy(ctx):
    _check(None, load_library().grpic_destroy(ctx), "grpic_destroy")


def grpic_step(ctx, nsteps):
    _check(ctx, load_library().grpic_step(ctx, int(nsteps)), "grpic_step")


def grpic_step_async(ctx, nsteps):
    _check(ctx, load_library().grpic_step_async(ctx, int(nsteps)), "grpic_step_async")


def grpic_sync(ctx):
    _check(ctx, load_library().grpic_sync(ctx), "grpic_sync")


def grpic_stage(ctx, stage):
    _check(ctx, load_library().grpic_stage(ctx, int(stage)), "grpic_stage")


def _is_cuda_tensor(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _as_arg(a, dtype):
    """(pointer, mem, keepalive) for a numpy array or a CUDA tensor."""
    if _is_cuda_tensor(a):
        t = a.contiguous().double() if dtype is np.float64 else a.contiguous()
        return ctypes.c_void_p(t.data_ptr()), GRPIC_MEM_DEVICE, t
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), GRPIC_MEM_HOST, arr


def grpic_set_fields(ctx, d3, b3):
    pd, md, kd = _as_arg(d3, np.float64)
    pb, mb, kb = _as_arg(b3, np.float64)
    assert md == mb
    _check(ctx, load_library().grpic_set_fields(ctx, pd, pb, md), "grpic_set_fields")


def grpic_set_uniform_field(ctx, E, B):
    e = (ctypes.c_double * 3)(*[float(v) for v in E])
    b = (ctypes.c_double * 3)(*[float(v) for v in B])
    _check(ctx, load_library().grpic_set_uniform_field(ctx, e, b), "grpic_set_uniform_field")


def grpic_set_j(ctx, J3):
    pj, mj, kj = _as_arg(J3, np.float64)
    _check(ctx, load_library().grpic_set_j(ctx, pj, mj), "grpic_set_j")


def grpic_load_particles(ctx, species, q_over_m, q_macro, x4, u4, ids, umode=GRPIC_U_FULL):
    n = int(x4.shape[1])
    px, mx, kx = _as_arg(x4, np.float64)
    pu, mu, ku = _as_arg(u4, np.float64)
    if _is_cuda_tensor(ids):
        ti = ids.contiguous()
        pi, mi, ki = ctypes.c_void_p(ti.data_ptr()), GRPIC_MEM_DEVICE, ti
    else:
        pi, mi, ki = _as_arg(ids, np.uint32)
    assert mx == mu == mi
    flags = int(umode) | (GRPIC_LOAD_DEVICE if mx == GRPIC_MEM_DEVICE else 0)
    _check(ctx, load_library().grpic_load_particles(ctx, int(species), float(q_over_m), float(q_macro), n, px, pu, pi,
                                                    flags), "grpic_load_particles")


def grpic_num_particles(ctx, species):
    n = ctypes.c_int64(0)
    _check(ctx, load_library().grpic_num_particles(ctx, int(species), ctypes.byref(n)), "grpic_num_particles")
    return n.value


def grpic_get_particles(ctx, species, device=False):
    """(x4, u4, ids) of a species: numpy arrays, or CUDA tensors (float64, float64, int32) with
    device=True (no host copy)."""
    n = grpic_num_particles(ctx, species)
    nn = ctypes.c_int64(n)
    if device:
        torch = _torch()
        x4 = torch.empty((4, n), dtype=torch.float64, device="cuda")
        u4 = torch.empty((4, n), dtype=torch.float64, device="cuda")
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        _check(ctx, load_library().grpic_get_particles(ctx, int(species), ctypes.byref(nn),
                                                       ctypes.c_void_p(x4.data_ptr()), ctypes.c_void_p(u4.data_ptr()),
                                                       ctypes.c_void_p(ids.data_ptr()), GRPIC_MEM_DEVICE),
               "grpic_get_particles")
        return x4[:, :nn.value], u4[:, :nn.value], ids[:nn.value]
    x4 = np.zeros((4, n))
    u4 = np.zeros((4, n))
    ids = np.zeros(n, dtype=np.uint32)
    _check(ctx, load_library().grpic_get_particles(ctx, int(species), ctypes.byref(nn),
                                                   x4.ctypes.data_as(ctypes.c_void_p),
                                                   u4.ctypes.data_as(ctypes.c_void_p),
                                                   ids.ctypes.data_as(ctypes.c_void_p), GRPIC_MEM_HOST),
           "grpic_get_particles")
    return x4[:, :nn.value], u4[:, :nn.value], ids[:nn.value]


def grpic_get_fields(ctx, shape):
    d = np.zeros((3,) + tuple(shape))
    b = np.zeros((3,) + tuple(shape))
    J = np.zeros((3,) + tuple(shape))
    _check(ctx, load_library().grpic_get_fields(ctx, d.ctypes.data_as(ctypes.c_void_p),
                                                b.ctypes.data_as(ctypes.c_void_p),
                                                J.ctypes.data_as(ctypes.c_void_p), GRPIC_MEM_HOST),
           "grpic_get_fields")
    return d, b, J


GRPIC_FIELD_D, GRPIC_FIELD_B, GRPIC_FIELD_J = 0, 1, 2


def grpic_get_fields_contra(ctx, shape):
    """(d, h): contravariant F^{i4} at the edges and (F^yz, F^zx, F^xy) at the faces, (3,) + shape each."""
    d = np.zeros((3,) + tuple(shape))
    h = np.zeros((3,) + tuple(shape))
    _check(ctx, load_library().grpic_get_fields_contra(ctx, d.ctypes.data_as(ctypes.c_void_p),
                                                       h.ctypes.data_as(ctypes.c_void_p), GRPIC_MEM_HOST),
           "grpic_get_fields_contra")
    return d, h


def grpic_get_planes(ctx, which, z0, nplanes, shape):
    """Planes z0 .. z0 + nplanes - 1 of field `which` (GRPIC_FIELD_D / _B / _J): a (3, nplanes, ny, nx)
    float64 array.  shape: the context's (nz, ny, nx)."""
    out = np.zeros((3, int(nplanes)) + tuple(shape[1:]))
    _check(ctx, load_library().grpic_get_planes(ctx, int(which), int(z0), int(nplanes),
                                                out.ctypes.data_as(ctypes.c_void_p), GRPIC_MEM_HOST),
           "grpic_get_planes")
    return out


def grpic_set_planes(ctx, which, z0, planes, add=False):
    """Write (or, for J with add, add into) planes z0 .. z0 + n - 1 of field `which` from a
    (3, n, ny, nx) array."""
    pa, mem, keep = _as_arg(planes, np.float64)
    n = int(planes.shape[1])
    _check(ctx, load_library().grpic_set_planes(ctx, int(which), int(z0), n, pa, mem, int(bool(add))),
           "grpic_set_planes")


def grpic_get_stats(ctx):
    s = grpic_stats()
    _check(ctx, load_library().grpic_get_stats(ctx, ctypes.byref(s)), "grpic_get_stats")
    return dict(steps=s.steps, removed_horizon=s.removed_horizon, removed_outer=s.removed_outer,
                gamma_fallbacks=s.gamma_fallbacks, fp64_evals=s.fp64_evals, particle_steps=s.particle_steps,
                n_alive=list(s.n_alive))


def grpic_set_profiling(ctx, on):
    _check(ctx, load_library().grpic_set_profiling(ctx, int(bool(on))), "grpic_set_profiling")


STAGE_NAMES = ("b_half", "zero_j", "push_deposit", "e_step", "sort", "b_half2")


def grpic_get_profile(ctx, reset=False):
    ms = (ctypes.c_double * 6)()
    cnt = (ctypes.c_int64 * 6)()
    nl = ctypes.c_int64(0)
    _check(ctx, load_library().grpic_get_profile(ctx, ms, cnt, ctypes.byref(nl), int(bool(reset))),
           "grpic_get_profile")
    return {STAGE_NAMES[q]: (ms[q], cnt[q]) for q in range(6)}, nl.value


def grpic_get_invariants(ctx, set_baseline=False):
    """Invariant statistics of the live particles (see include/grpic.h) as a dict."""
    out = grpic_invariants()
    _check(ctx, load_library().grpic_get_invariants(ctx, int(bool(set_baseline)), ctypes.byref(out)),
           "grpic_get_invariants")
    return {k: getattr(out, k) for k, _ in grpic_invariants._fields_}


def grpic_charge_density(ctx, shape, with_gamma=False):
    """(nz, ny, nx) float64 charge density at the nodes (J^4 / c with with_gamma)."""
    rho = np.zeros(shape)
    _check(ctx, load_library().grpic_charge_density(ctx, int(bool(with_gamma)), rho.ctypes.data_as(ctypes.c_void_p),
                                                    GRPIC_MEM_HOST), "grpic_charge_density")
    return rho


def grpic_gauss_residual(ctx, shape=None):
    """(residual field or None, max |residual| over [2, n-3]^3)."""
    mx = ctypes.c_double(0.0)
    res = np.zeros(shape) if shape is not None else None
    _check(ctx, load_library().grpic_gauss_residual(ctx, None if res is None else res.ctypes.data_as(ctypes.c_void_p),
                                                    GRPIC_MEM_HOST, ctypes.byref(mx)), "grpic_gauss_residual")
    return res, mx.value


def grpic_set_tuning(ctx, far_min_blocks, near_blocks_per_sm, sort_interval, overlap=1, split=0, j_tile=0,
                     spread=0, area_table=0):
    t = grpic_tuning(int(far_min_blocks), int(near_blocks_per_sm), int(sort_interval), int(overlap), int(split),
                     int(j_tile), int(spread), int(area_table))
    _check(ctx, load_library().grpic_set_tuning(ctx, ctypes.byref(t)), "grpic_set_tuning")


def grpic_get_tuning(ctx):
    t = grpic_tuning()
    _check(ctx, load_library().grpic_get_tuning(ctx, ctypes.byref(t)), "grpic_get_tuning")
    return dict(far_min_blocks=t.far_min_blocks, near_blocks_per_sm=t.near_blocks_per_sm,
                sort_interval=t.sort_interval, overlap=t.overlap, split=t.split, j_tile=t.j_tile,
                spread=t.spread, area_table=t.area_table)


def grpic_check_newton64(n=1 << 22):
    out = (ctypes.c_double * 3)()
    _check(None, load_library().grpic_check_newton64(int(n), out), "grpic_check_newton64")
    return dict(rcp=out[0], div=out[1], sqrt=out[2])


def grpic_check_conversions(n=1 << 24):
    out = (ctypes.c_int64 * 2)()
    _check(None, load_library().grpic_check_conversions(int(n), out), "grpic_check_conversions")
    return dict(widen=out[0], narrow=out[1])


def grpic_probe_fma_peak(precision):
    v = ctypes.c_double(0.0)
    _check(None, load_library().grpic_probe_fma_peak(int(precision), ctypes.byref(v)), "grpic_probe_fma_peak")
    return v.value


def grpic_sort_particles_static(nx, ny, nz, x4, u4, ids, x4_out, u4_out, ids_out, n_out, stream=None):
    """Cell sort that allocates nothing (see include/grpic.h).  All array arguments are CUDA
    tensors: x4/u4 (4, n) float64, ids (n,) int32 or uint32, outputs of the same shapes, n_out a
    one-element int64 tensor.  Runs on `stream` (default: PyTorch's current stream)."""
    if stream is None:
        stream = _torch().cuda.current_stream().cuda_stream
    n = int(x4.shape[1])
    for t in (x4, u4, ids, x4_out, u4_out, ids_out, n_out):
        assert _is_cuda_tensor(t) and t.is_contiguous()
    code = load_library().grpic_sort_particles_static(
        int(nx), int(ny), int(nz), n, x4.data_ptr(), u4.data_ptr(), ids.data_ptr(), x4_out.data_ptr(),
        u4_out.data_ptr(), ids_out.data_ptr(), n_out.data_ptr(), ctypes.c_void_p(stream))
    if code != GRPIC_OK:
        raise GrpicError(code, "grpic_sort_particles_static",
                         "grid larger than 64^3 cells or n >= 2^31" if code == 8 else "")


def grpic_batch_create(ctxs, stream=None):
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    h = ctypes.c_void_p()
    _check(None, load_library().grpic_batch_create(arr, len(ctxs), stream, ctypes.byref(h)), "grpic_batch_create")
    return h.value


def grpic_batch_step(b, nsteps):
    _check(None, load_library().grpic_batch_step(b, int(nsteps)), "grpic_batch_step")


def grpic_batch_info(b):
    k = ctypes.c_int64(0)
    w = ctypes.c_int64(0)
    _check(None, load_library().grpic_batch_info(b, ctypes.byref(k), ctypes.byref(w)), "grpic_batch_info")
    return k.value, w.value


def grpic_batch_set_blocks_per_sm(b, blocks_per_sm):
    _check(None, load_library().grpic_batch_set_blocks_per_sm(b, int(blocks_per_sm)),
           "grpic_batch_set_blocks_per_sm")


def grpic_batch_destroy(b):
    _check(None, load_library().grpic_batch_destroy(b), "grpic_batch_destroy")


def grpic_server_create(hbm_budget, max_slots, torch_allocator=True):
    h = ctypes.c_void_p()
    alloc, free = (_torch_alloc, _torch_free) if torch_allocator else (ALLOC_FN(), FREE_FN())
    _check(None, load_library().grpic_server_create(int(hbm_budget), int(max_slots), alloc, free, None,
                                                    ctypes.byref(h)), "grpic_server_create")
    return h.value


def grpic_submit(server, req):
    t = ctypes.c_uint64(0)
    _check(None, load_library().grpic_submit(server, ctypes.byref(req), ctypes.byref(t)), "grpic_submit")
    return t.value


def grpic_server_tick(server):
    r = ctypes.c_int(0)
    q = ctypes.c_int(0)
    _check(None, load_library().grpic_server_tick(server, ctypes.byref(r), ctypes.byref(q)), "grpic_server_tick")
    return r.value, q.value


def grpic_poll(server, ticket, with_status=False):
    """(state, ctx handle or None); raises if the finished run failed, unless with_status, which
    returns (state, ctx, status) instead (status GRPIC_OK, or the run's own error)."""
    st = ctypes.c_int(0)
    ctx = ctypes.c_void_p()
    code = load_library().grpic_poll(server, int(ticket), ctypes.byref(st), ctypes.byref(ctx))
    if with_status:
        return st.value, ctx.value, (GRPIC_OK if code == 7 else code)
    if code not in (GRPIC_OK, 7):
        raise GrpicError(code, "grpic_poll")
    return st.value, ctx.value


def grpic_server_release(server, ticket):
    _check(None, load_library().grpic_server_release(server, int(ticket)), "grpic_server_release")


def grpic_request_bytes(req):
    b = ctypes.c_size_t(0)
    _check(None, load_library().grpic_request_bytes(ctypes.byref(req), ctypes.byref(b)), "grpic_request_bytes")
    return b.value


def grpic_server_destroy(server):
    _check(None, load_library().grpic_server_destroy(server), "grpic_server_destroy")


def make_request(n, m, a, ppc, nsteps, seed, precision="fp32_mixed", c=1.0, dt=0.4, B=(0.0, 0.0, 0.05),
                 species=((-1.0,), (1.0,)), wp_dt=0.025, u_th=0.1, r_min=None, quad_order=2, absorb_inner=0.0,
                 absorb_outer=0.0, absorb_width=0):
    """A run request: n^3 grid, pair plasma (q/m = -1, +1) by default, macro charge for the
    stated omega_p dt at ppc particles per cell per species (0.025 by default: charge separation
    near the hole stays bounded over 500 steps there, larger values overshoot the step limit)."""
    prec = {"fp64": GRPIC_FP64, "fp32_mixed": GRPIC_FP32_MIXED}[precision]
    qms = [sp[0] for sp in species]
    q = (wp_dt / dt) ** 2 / (4.0 * np.pi * max(ppc, 1) * sum(abs(v) for v in qms))
    req = grpic_request()
    req.cfg = grpic_config(n, n, n, m, a, c, dt, prec, quad_order, 0.0, 0, 1, 0, 0.0, absorb_inner, absorb_outer,
                           absorb_width)
    req.B_contra[:] = list(B)
    req.nspecies = len(qms)
    for s_, qm in enumerate(qms):
        req.q_over_m[s_] = qm
        req.q_macro[s_] = float(np.sign(qm) * q)
    req.ppc = ppc
    req.u_th = u_th
    req.r_min = 2.5 * m if r_min is None else r_min
    req.seed = seed
    req.nsteps = nsteps
    return req


# ---- convenience wrapper -----------------------------------------------------------------------
class Simulation:
    """One GRPIC context on the current CUDA device and PyTorch's current stream."""

    def __init__(self, nx, ny, nz, m, a, c, dt, precision="fp64", quad_order=2, r_excise=0.0, flags=0,
                 sort_interval=1, max_particles=0, stream=None, torch_allocator=True, fp64_radius=0.0,
                 absorb_inner=0.0, absorb_outer=0.0, absorb_width=0, z_origin=0, nz_total=0):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("GRPIC needs a CUDA device")
        load_library()
        self.shape = (nz, ny, nx)
        prec = {"fp64": GRPIC_FP64, "fp32_mixed": GRPIC_FP32_MIXED}[precision]
        cfg = grpic_config(nx, ny, nz, m, a, c, dt, prec, quad_order, r_excise, flags, sort_interval, max_particles,
                           fp64_radius, absorb_inner, absorb_outer, absorb_width, z_origin, nz_total)
        if torch_allocator:
            cfg.alloc = _torch_alloc
            cfg.free_fn = _torch_free
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.handle = grpic_create(cfg, ctypes.c_void_p(stream))
        self.precision = precision

    def close(self):
        if getattr(self, "handle", None):
            grpic_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, d, b):
        grpic_set_fields(self.handle, d, b)

    def set_uniform_field(self, E=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0)):
        grpic_set_uniform_field(self.handle, E, B)

    def set_j(self, J):
        grpic_set_j(self.handle, J)

    def load_particles(self, species, q_over_m, q_macro, x4, u4, ids, umode=GRPIC_U_FULL):
        if u4.shape[0] == 3:
            u4 = np.vstack([np.asarray(u4), np.zeros((1, u4.shape[1]))])
        grpic_load_particles(self.handle, species, q_over_m, q_macro, x4, u4, ids, umode)

    def step(self, n=1):
        grpic_step(self.handle, n)

    def step_async(self, n=1):
        grpic_step_async(self.handle, n)

    def sync(self):
        grpic_sync(self.handle)

    def stage(self, s):
        grpic_stage(self.handle, s)

    def get_fields(self):
        return grpic_get_fields(self.handle, self.shape)

    def get_particles(self, species, device=False):
        return grpic_get_particles(self.handle, species, device=device)

    def get_fields_contra(self):
        return grpic_get_fields_contra(self.handle, self.shape)

    def get_planes(self, which, z0, nplanes):
        return grpic_get_planes(self.handle, which, z0, nplanes, self.shape)

    def set_planes(self, which, z0, planes, add=False):
        grpic_set_planes(self.handle, which, z0, planes, add)

    def num_particles(self, species):
        return grpic_num_particles(self.handle, species)

    def stats(self):
        return grpic_get_stats(self.handle)

    def set_profiling(self, on=True):
        grpic_set_profiling(self.handle, on)

    def profile(self, reset=False):
        return grpic_get_profile(self.handle, reset)

    def set_tuning(self, far_min_blocks=4, near_blocks_per_sm=4, sort_interval=1, overlap=1, split=0, j_tile=0,
                   spread=1, area_table=0):
        grpic_set_tuning(self.handle, far_min_blocks, near_blocks_per_sm, sort_interval, overlap, split, j_tile,
                         spread, area_table)

    def tuning(self):
        return grpic_get_tuning(self.handle)

    def invariants(self, baseline=False):
        return grpic_get_invariants(self.handle, baseline)

    def charge_density(self, with_gamma=False):
        return grpic_charge_density(self.handle, self.shape, with_gamma)

    def gauss_residual(self, field=True):
        return grpic_gauss_residual(self.handle, self.shape if field else None)
