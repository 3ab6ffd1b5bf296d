"""GRPIC oracle -- TEST INFRASTRUCTURE ONLY.

Python face of ``oracle/grpic_oracle.cpp``: a plain, slow FP64 CPU implementation of the
GRPIC timestep of Watson & Nishikawa (arXiv:0904.0232), written from the paper and sharing
no code with the CUDA library.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import it.

Grid arrays are ``(3, nz, ny, nx)`` float64 (component, then z-major); particle arrays are
planar ``(4, n)`` float64 (x^1, x^2, x^3, x^4 and u^1..u^4).  Component order of the
prognostic field: ``d = (F^{x4}, F^{y4}, F^{z4})`` (contravariant, on edges) and
``b = (F_{yz}, F_{zx}, F_{xy})`` (covariant, on faces).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grpic_oracle.cpp")
_LIB = os.path.join(_HERE, "libgrpic_oracle.so")
_lock = threading.Lock()
_lib = None

NO_GAMMA_IN_J = 1
NO_GAMMA_TERMS = 2
FROZEN_FIELDS = 4
LITERAL_HALF_STEPS = 8
RK4_AS_PRINTED = 16  # ablation only: the printed RK4 steps (Sec. 3.3) with x_n, u_n added to the finals
ANALYTIC_WALD = 32  # test-particle pins only: the Lorentz term of Eq. 15 takes Wald's field at the particle

OK, ERR_INVALID, ERR_CFL, ERR_NONFINITE = 0, 1, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle (plain g++, -O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("m", ctypes.c_double), ("a", ctypes.c_double), ("c", ctypes.c_double),
                ("dt", ctypes.c_double), ("quad_order", ctypes.c_int),
                ("r_excise", ctypes.c_double), ("flags", ctypes.c_uint), ("threads", ctypes.c_int),
                ("absorb_inner", ctypes.c_double), ("absorb_outer", ctypes.c_double), ("absorb_width", ctypes.c_int),
                ("z_origin", ctypes.c_int), ("nz_total", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_LL = ctypes.POINTER(ctypes.c_longlong)
_V = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_kerr_r": (ctypes.c_double, [_D, ctypes.c_double]),
                "orc_kerr_fk": (None, [_D, ctypes.c_double, ctypes.c_double, _D]),
                "orc_metric": (None, [_D, ctypes.c_double, ctypes.c_double, _D]),
                "orc_metric_inverse": (ctypes.c_int, [_D, ctypes.c_double, ctypes.c_double, _D]),
                "orc_metric_det": (ctypes.c_double, [_D, ctypes.c_double, ctypes.c_double]),
                "orc_metric_grad": (None, [_D, ctypes.c_double, ctypes.c_double, _D]),
                "orc_christoffel": (None, [_D, ctypes.c_double, ctypes.c_double, _D]),
                "orc_gamma_from_v": (ctypes.c_double, [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]),
                "orc_gamma_f": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I]),
                "orc_solve_u4": (ctypes.c_int, [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, ctypes.c_int, _D]),
                "orc_complete_tensor": (ctypes.c_int, [_D, _D, _D, _D, _D]),
                "orc_gauss_legendre": (None, [ctypes.c_int, _D, _D]),
                "orc_volume_weights": (None, [_D, _I, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]),
                "orc_wald_field": (None, [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]),
                "orc_create": (_V, [ctypes.POINTER(_Cfg)]),
                "orc_destroy": (None, [_V]),
                "orc_r_plus": (ctypes.c_double, [_V]),
                "orc_set_fields": (ctypes.c_int, [_V, _D, _D]),
                "orc_set_absorb_target": (ctypes.c_int, [_V, _D, _D]),
                "orc_get_contra_h": (ctypes.c_int, [_V, _D]),
                "orc_absorb_kappa": (ctypes.c_double, [_V, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_set_j": (ctypes.c_int, [_V, _D]),
                "orc_get_fields": (ctypes.c_int, [_V, _D, _D, _D]),
                "orc_init_uniform_field": (ctypes.c_int, [_V, _D, _D]),
                "orc_init_wald": (ctypes.c_int, [_V, ctypes.c_double]),
                "orc_load_particles": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_longlong, _D, _D, _U32, ctypes.c_int]),
                "orc_num_particles": (ctypes.c_longlong, [_V, ctypes.c_int]),
                "orc_get_particles": (ctypes.c_int, [_V, ctypes.c_int, _D, _D, _U32]),
                "orc_step": (ctypes.c_int, [_V, ctypes.c_int]),
                "orc_stage_b_half": (ctypes.c_int, [_V]),
                "orc_stage_b_half2": (ctypes.c_int, [_V]),
                "orc_stage_e": (ctypes.c_int, [_V]),
                "orc_stage_zero_j": (ctypes.c_int, [_V]),
                "orc_stage_push_deposit": (ctypes.c_int, [_V]),
                "orc_accel": (ctypes.c_int, [_V, ctypes.c_double, _D, _D, _D]),
                "orc_gather": (ctypes.c_int, [_V, ctypes.c_int, _D, _D]),
                "orc_set_wald_b0": (None, [_V, ctypes.c_double]),
                "orc_deposit": (ctypes.c_int, [_V, _D, _D, ctypes.c_double, ctypes.c_double]),
                "orc_face_weights": (None, [_V, ctypes.c_int, _D, _I, _D]),
                "orc_get_stats": (None, [_V, _LL]),
                "orc_last_moves": (ctypes.c_int, [_V, ctypes.c_int, _LL, _D, _D, _U32]),
                "orc_gamma_terms": (None, [_V, _D]),
                "orc_max_threads": (ctypes.c_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ----------------------------------------------------------------------------------------
# Pointwise functions (positions X are relative to the central mass).
# ----------------------------------------------------------------------------------------
def kerr_r(X, a):
    """Non-negative root of Eq. 6."""
    return lib().orc_kerr_r(_dp(_f64(X)), float(a))


def kerr_fk(X, m, a):
    """(r, f, k_mu) of Eqs. 4-6: g = eta + f k k."""
    out = np.zeros(6)
    lib().orc_kerr_fk(_dp(_f64(X)), float(m), float(a), _dp(out))
    return out[0], out[1], out[2:6].copy()


def metric(X, m, a):
    """g_{mu nu} of Eq. 4 (4x4; index 3 = x^4 = c t)."""
    g = np.zeros(16)
    lib().orc_metric(_dp(_f64(X)), float(m), float(a), _dp(g))
    return g.reshape(4, 4)


def metric_inverse(X, m, a):
    gi = np.zeros(16)
    if lib().orc_metric_inverse(_dp(_f64(X)), float(m), float(a), _dp(gi)) != OK:
        raise ValueError("singular metric")
    return gi.reshape(4, 4)


def metric_det(X, m, a):
    return lib().orc_metric_det(_dp(_f64(X)), float(m), float(a))


def metric_grad(X, m, a):
    """dg[l, mu, nu] = d_l g_{mu nu} for l = x, y, z (dual numbers)."""
    dg = np.zeros(48)
    lib().orc_metric_grad(_dp(_f64(X)), float(m), float(a), _dp(dg))
    return dg.reshape(3, 4, 4)


def christoffel(X, m, a):
    """G[al, mu, nu] = Gamma^al_{mu nu}."""
    G = np.zeros(64)
    lib().orc_christoffel(_dp(_f64(X)), float(m), float(a), _dp(G))
    return G.reshape(4, 4, 4)


def gamma_from_v(X, m, a, c, v3):
    """Eq. 7: Lorentz factor from the coordinate velocity v^i = dx^i/dt."""
    return lib().orc_gamma_from_v(_dp(_f64(X)), float(m), float(a), float(c), _dp(_f64(v3)))


def gamma_f(u4, a4, c, dt):
    """Eq. 16; returns (gamma, fallback_used)."""
    fb = ctypes.c_int(0)
    g = lib().orc_gamma_f(float(u4), float(a4), float(c), float(dt), ctypes.byref(fb))
    return g, bool(fb.value)


def solve_u4(X, m, a, c, usp, mode):
    """Future-directed unit 4-velocity from spatial components: mode 1 covariant u_i,
    mode 2 contravariant u^i."""
    u = np.zeros(4)
    if lib().orc_solve_u4(_dp(_f64(X)), float(m), float(a), float(c), _dp(_f64(usp)), int(mode), _dp(u)) != OK:
        raise ValueError("no future-directed solution")
    return u


def complete_tensor(g, b, d):
    """Full contravariant and covariant field tensor from covariant F_{yz},F_{zx},F_{xy} = b and
    contravariant F^{x4},F^{y4},F^{z4} = d, with metric g at that point."""
    Fu = np.zeros(16)
    Fd = np.zeros(16)
    if lib().orc_complete_tensor(_dp(_f64(g).ravel()), _dp(_f64(b)), _dp(_f64(d)), _dp(Fu), _dp(Fd)) != OK:
        raise ValueError("singular conversion")
    return Fu.reshape(4, 4), Fd.reshape(4, 4)


def gauss_legendre(Q):
    x = np.zeros(Q)
    w = np.zeros(Q)
    lib().orc_gauss_legendre(int(Q), _dp(x), _dp(w))
    return x, w


def volume_weights(P, cell, Xc, m, a, Q):
    """Sec. 3.3 CIC weights with sub-volumes integrated literally (sqrt(-det g))."""
    W = np.zeros(8)
    c = np.ascontiguousarray(cell, dtype=np.int32)
    lib().orc_volume_weights(_dp(_f64(P)), c.ctypes.data_as(_I), _dp(_f64(Xc)), float(m), float(a), int(Q), _dp(W))
    return W


def wald_field(X, m, a, B0):
    """(F_{mn}, F^{mn}) of the Wald vacuum field A = (B0/2)(xi_phi + 2 a xi_t)."""
    Fd = np.zeros(16)
    Fu = np.zeros(16)
    lib().orc_wald_field(_dp(_f64(X)), float(m), float(a), float(B0), _dp(Fd), _dp(Fu))
    return Fd.reshape(4, 4), Fu.reshape(4, 4)


def max_threads():
    return lib().orc_max_threads()


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class Oracle:
    """One oracle simulation context (grid, metric, fields, particles)."""

    def __init__(self, nx, ny, nz, m, a, c, dt, quad_order=2, r_excise=0.0, flags=0, threads=1, absorb_inner=0.0,
                 absorb_outer=0.0, absorb_width=0, z_origin=0, nz_total=0):
        self.shape = (nz, ny, nx)
        self.ncell = nx * ny * nz
        cfg = _Cfg(nx, ny, nz, m, a, c, dt, quad_order, r_excise, flags, threads, absorb_inner, absorb_outer,
                   absorb_width, z_origin, nz_total)
        self._h = lib().orc_create(ctypes.byref(cfg))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        self.cfg = dict(nx=nx, ny=ny, nz=nz, m=m, a=a, c=c, dt=dt, quad_order=quad_order,
                        r_excise=r_excise, flags=flags, threads=threads, absorb_inner=absorb_inner,
                        absorb_outer=absorb_outer, absorb_width=absorb_width, z_origin=z_origin,
                        nz_total=nz_total)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, code, what):
        if code != OK:
            raise OracleError(code, what)

    @property
    def r_plus(self):
        return lib().orc_r_plus(self._h)

    @property
    def centre(self):
        nzt = self.cfg["nz_total"] or self.cfg["nz"]
        return np.array([(self.cfg["nx"] - 1) / 2, (self.cfg["ny"] - 1) / 2, (nzt - 1) / 2 - self.cfg["z_origin"]])

    def set_fields(self, d, b):
        d = _f64(d, (3,) + self.shape)
        b = _f64(b, (3,) + self.shape)
        self._chk(lib().orc_set_fields(self._h, _dp(d), _dp(b)), "set_fields")

    def set_absorb_target(self, d, b):
        """Replace the absorbing layers' target (reading A23; by default the field as last set)."""
        d = _f64(d, (3,) + self.shape)
        b = _f64(b, (3,) + self.shape)
        self._chk(lib().orc_set_absorb_target(self._h, _dp(d), _dp(b)), "set_absorb_target")

    def absorb_kappa(self, comp, i, j, k):
        """Relaxation per step of the absorbing layers at component comp's point (i, j, k) (A23)."""
        return lib().orc_absorb_kappa(self._h, int(comp), int(i), int(j), int(k))

    def set_j(self, J):
        J = _f64(J, (3,) + self.shape)
        self._chk(lib().orc_set_j(self._h, _dp(J)), "set_j")

    def get_fields(self):
        d = np.zeros((3,) + self.shape)
        b = np.zeros((3,) + self.shape)
        J = np.zeros((3,) + self.shape)
        self._chk(lib().orc_get_fields(self._h, _dp(d), _dp(b), _dp(J)), "get_fields")
        return d, b, J

    def get_contra_h(self):
        """Contravariant (F^yz, F^zx, F^xy) at the b faces from the current (b, d), as the E step
        converts them; zero on the outer index layer."""
        h = np.zeros((3,) + self.shape)
        self._chk(lib().orc_get_contra_h(self._h, _dp(h)), "get_contra_h")
        return h

    def init_uniform_field(self, E=(0.0, 0.0, 0.0), B=(0.0, 0.0, 0.0)):
        self._chk(lib().orc_init_uniform_field(self._h, _dp(_f64(E)), _dp(_f64(B))), "init_uniform_field")

    def init_wald(self, B0):
        self._chk(lib().orc_init_wald(self._h, float(B0)), "init_wald")

    def load_particles(self, species, q_over_m, q_macro, x4, u4, ids, umode=0):
        x4 = _f64(x4)
        u4 = _f64(u4)
        n = x4.shape[1]
        assert x4.shape == (4, n) and u4.shape[1] == n
        if u4.shape[0] == 3:
            u4 = np.vstack([u4, np.zeros((1, n))])
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        self._chk(lib().orc_load_particles(self._h, int(species), float(q_over_m), float(q_macro), n,
                                           _dp(x4), _dp(u4), ids.ctypes.data_as(_U32), int(umode)),
                  "load_particles")

    def num_particles(self, species):
        return int(lib().orc_num_particles(self._h, int(species)))

    def get_particles(self, species):
        n = self.num_particles(species)
        x4 = np.zeros((4, n))
        u4 = np.zeros((4, n))
        ids = np.zeros(n, dtype=np.uint32)
        self._chk(lib().orc_get_particles(self._h, int(species), _dp(x4), _dp(u4), ids.ctypes.data_as(_U32)),
                  "get_particles")
        return x4, u4, ids

    def step(self, nsteps=1):
        self._chk(lib().orc_step(self._h, int(nsteps)), "step")

    def b_half(self):
        """First B half-step (b^{n-1/2} -> b^n)."""
        self._chk(lib().orc_stage_b_half(self._h), "b_half")

    def b_half2(self):
        """Second B half-step (-> b^{n+1/2})."""
        self._chk(lib().orc_stage_b_half2(self._h), "b_half2")

    def e_step(self):
        self._chk(lib().orc_stage_e(self._h), "e_step")

    def zero_j(self):
        self._chk(lib().orc_stage_zero_j(self._h), "zero_j")

    def push_deposit(self):
        self._chk(lib().orc_stage_push_deposit(self._h), "push_deposit")

    def accel(self, q_over_m, x4, u4):
        out = np.zeros(4)
        self._chk(lib().orc_accel(self._h, float(q_over_m), _dp(_f64(x4)), _dp(_f64(u4)), _dp(out)), "accel")
        return out

    def gather(self, comp, x3):
        """CIC value of prognostic component comp (0..2 = d, 3..5 = b) at grid position x3."""
        out = np.zeros(1)
        self._chk(lib().orc_gather(self._h, int(comp), _dp(_f64(x3)), _dp(out)), "gather")
        return float(out[0])

    def set_wald_b0(self, B0):
        """Field strength of Wald's field for a context created with ANALYTIC_WALD."""
        lib().orc_set_wald_b0(self._h, float(B0))

    def deposit(self, x1, x2, q_macro, gbar=1.0):
        self._chk(lib().orc_deposit(self._h, _dp(_f64(x1)), _dp(_f64(x2)), float(q_macro), float(gbar)), "deposit")

    def face_weights(self, K, P, cell):
        W = np.zeros(4)
        c = np.ascontiguousarray(cell, dtype=np.int32)
        lib().orc_face_weights(self._h, int(K), _dp(_f64(P)), c.ctypes.data_as(_I), _dp(W))
        return W

    def last_moves(self, species):
        """(x0, x1, ids) of every particle of the last push, removed ones included."""
        n = ctypes.c_longlong(0)
        self._chk(lib().orc_last_moves(self._h, int(species), ctypes.byref(n), None, None, None), "last_moves")
        x0 = np.zeros((3, n.value))
        x1 = np.zeros((3, n.value))
        ids = np.zeros(n.value, dtype=np.uint32)
        self._chk(lib().orc_last_moves(self._h, int(species), ctypes.byref(n), _dp(x0), _dp(x1),
                                       ids.ctypes.data_as(_U32)), "last_moves")
        return x0, x1, ids

    def stats(self):
        out = (ctypes.c_longlong * 4)()
        lib().orc_get_stats(self._h, out)
        return dict(removed_horizon=out[0], removed_outer=out[1], f_fallbacks=out[2], steps=out[3])

    def gamma_terms(self):
        out = np.zeros(2)
        lib().orc_gamma_terms(self._h, _dp(out))
        return out[0], out[1]
