"""Operation count of one GRPIC particle-step -- TEST AND MEASUREMENT INFRASTRUCTURE ONLY.

The roofline of the push kernel divides an algorithmic operation count per particle-step by the
kernel's time.  This module fixes that count by running a plain restatement of the method's
arithmetic on a counting scalar: every add, subtract, multiply, divide and square root of one
particle-step is counted once (a fused multiply-add is two operations; comparisons, floors,
minima and maxima, and constants of a whole run are not counted).  The restatement takes the
closed forms the method is built from, each written the straightforward way:

* Kerr metric at a point (Eqs. 4-6): the quartic's non-negative root r, f = 2 m r^3 / Sigma,
  k = ((r x - a y)/(r^2 + a^2), (r y + a x)/(r^2 + a^2), z / r);
* Christoffel contraction Gamma^a_mn u^m u^n for g = eta + f k k in closed form (gradients of r,
  f and k from the quartic by the chain rule);
* CIC gather (Sec. 3.3): per component eight trilinear weights about its own Yee lattice and
  their weighted sum;
* the tensor at the particle from (b, d) (Eq. 8 solved for F^{jk}), Lorentz term (q/m) F^a_b u^b
  (Eq. 15) and a~ = Lorentz - Christoffel;
* classical RK4 in proper time with one step h = dt / gamma_1 (Eqs. 13-16, reading A1);
* Umeda's zig-zag split and, per segment and direction, the four sub-areas of Eq. 18 by Q x Q
  Gauss-Legendre with the integrand sqrt(1 + f (k_I^2 + k_J^2)) from the quartic at each node,
  the weights, and the four flux contributions (J = rho gamma v, reading A13);
* the removal test r <= r_+ (Sec. 5 of the readings).

The particle-step it computes is checked against the oracle's (tests/test_flop_count.py), so the
count belongs to arithmetic that produces the method's result.  It is the numerator of the push
kernel's roofline; the kernels evaluate the same quantities with fewer operations (shared
reciprocals, factored lattices), which makes them faster but does not change this count.
"""
from __future__ import annotations

import math

import numpy as np


class Counter:
    def __init__(self):
        self.n = 0


_C = Counter()


class F:
    """A float64 whose arithmetic is counted."""

    __slots__ = ("v",)

    def __init__(self, v):
        self.v = float(v.v if isinstance(v, F) else v)

    @staticmethod
    def _w(o):
        return o.v if isinstance(o, F) else float(o)

    def __add__(self, o):
        _C.n += 1
        return F(self.v + F._w(o))

    __radd__ = __add__

    def __sub__(self, o):
        _C.n += 1
        return F(self.v - F._w(o))

    def __rsub__(self, o):
        _C.n += 1
        return F(F._w(o) - self.v)

    def __mul__(self, o):
        _C.n += 1
        return F(self.v * F._w(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        _C.n += 1
        return F(self.v / F._w(o))

    def __rtruediv__(self, o):
        _C.n += 1
        return F(F._w(o) / self.v)

    def __neg__(self):
        return F(-self.v)  # a sign change is not an operation

    def __float__(self):
        return self.v


def sqrt(x):
    _C.n += 1
    return F(math.sqrt(x.v))


def val(x):
    return x.v if isinstance(x, F) else float(x)


# Yee offsets (half cells) of the prognostic components: d^x, d^y, d^z on edges; b_x, b_y, b_z on faces
_YEE = ((1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0))


class Run:
    """Constants of a run (not counted): grid, centre, m, a, c, dt, Q and the Gauss-Legendre rule."""

    def __init__(self, shape, m, a, c, dt, quad_order=2):
        self.nz, self.ny, self.nx = shape
        self.cen = ((self.nx - 1) / 2.0, (self.ny - 1) / 2.0, (self.nz - 1) / 2.0)
        self.m, self.a, self.c, self.dt = m, a, c, dt
        self.a2 = a * a
        self.two_m = 2.0 * m
        self.r_plus = m + math.sqrt(max(0.0, m * m - a * a))
        x, w = np.polynomial.legendre.leggauss(quad_order)
        self.gx, self.gw = [float(v) for v in x], [float(v) for v in w]

    # ---- Eqs. 4-6 ------------------------------------------------------------------------
    def metric(self, X, Y, Z):
        R2 = X * X + Y * Y + Z * Z
        p = R2 - self.a2
        q = self.a2 * (Z * Z)
        D = sqrt(p * p + 4.0 * q)
        r2 = 0.5 * (p + D) if val(p) >= 0.0 else (2.0 * q) / (D - p)
        r = sqrt(r2)
        sig = r2 * r2 + q
        f = self.two_m * r * r2 / sig
        rho2 = r2 + self.a2
        k = ((r * X - self.a * Y) / rho2, (r * Y + self.a * X) / rho2, Z / r)
        return dict(r=r, r2=r2, D=D, sig=sig, f=f, k=k, rho2=rho2)

    # ---- Gamma^a_mn u^m u^n in closed form --------------------------------------------------
    def christoffel_uu(self, M, X, Y, Z, u):
        r, r2, D, sig, f, (k0, k1, k2), rho2 = M["r"], M["r2"], M["D"], M["sig"], M["f"], M["k"], M["rho2"]
        a, a2 = self.a, self.a2
        # grad r from the quartic: r_x = x r / D, r_y = y r / D, r_z = z (r^2 + a^2) / (r D)
        rx = X * r / D
        ry = Y * r / D
        rz = Z * rho2 / (r * D)
        # grad f: df/dr = f (3/r - 4 r^3 / Sigma), df/dz|_r = -2 a^2 z f / Sigma
        fr = f * (3.0 / r - 4.0 * r2 * r / sig)
        fg = (fr * rx, fr * ry, fr * rz - 2.0 * a2 * Z * f / sig)
        ri = (rx, ry, rz)
        xv = (X, Y, Z)
        # J[i][j] = d_i k_j
        Jk = []
        for i in range(3):
            tr = 2.0 * r * ri[i]
            j0 = xv[0] * ri[i] - tr * k0
            j1 = xv[1] * ri[i] - tr * k1
            if i == 0:
                j0 = j0 + r
                j1 = j1 + a
            elif i == 1:
                j0 = j0 - a
                j1 = j1 + r
            j2 = (1.0 - k2 * ri[i]) if i == 2 else (-(k2 * ri[i]))
            Jk.append((j0 / rho2, j1 / rho2, j2 / r))
        kv = (k0, k1, k2)
        s = k0 * u[0] + k1 * u[1] + k2 * u[2] + u[3]
        uf = u[0] * fg[0] + u[1] * fg[1] + u[2] * fg[2]
        Dv = [u[0] * Jk[0][j] + u[1] * Jk[1][j] + u[2] * Jk[2][j] for j in range(3)]
        Ev = [u[0] * Jk[j][0] + u[1] * Jk[j][1] + u[2] * Jk[j][2] for j in range(3)]
        uD = u[0] * Dv[0] + u[1] * Dv[1] + u[2] * Dv[2]
        c1 = uf * s + f * uD
        fs = f * s
        hs2 = 0.5 * s * s
        w = [c1 * kv[j] + fs * (Dv[j] - Ev[j]) - hs2 * fg[j] for j in range(3)]
        kw = k0 * w[0] + k1 * w[1] + k2 * w[2] - c1
        return [w[0] - f * k0 * kw, w[1] - f * k1 * kw, w[2] - f * k2 * kw, f * kw - c1]

    # ---- CIC gather (Sec. 3.3): eight trilinear weights per component ----------------------
    def gather(self, fields, x):
        out = []
        frac = {}
        for ax in range(3):
            for hh in (0, 1):
                s = x[ax] - 0.5 if hh else x[ax]
                i0 = int(math.floor(val(s)))
                frac[(ax, hh)] = (i0, s - float(i0))
        for comp in range(6):
            (ix, fx), (iy, fy), (iz, fz) = (frac[(ax, _YEE[comp][ax])] for ax in range(3))
            gx, gy, gz = 1.0 - fx, 1.0 - fy, 1.0 - fz
            wxy = (gx * gy, fx * gy, gx * fy, fx * fy)
            arr = fields[comp]
            acc = None
            for dz in (0, 1):
                wz = fz if dz else gz
                for n, (dx, dy) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
                    term = (wxy[n] * wz) * float(arr[iz + dz, iy + dy, ix + dx])
                    acc = term if acc is None else acc + term
            out.append(acc)
        return out[:3], out[3:]

    # ---- a~ = (q/m) F^a_b u^b - Gamma u u (Eqs. 8, 15) -------------------------------------
    def accel(self, fields, x, u, qm):
        d, b = self.gather(fields, x)
        X, Y, Z = x[0] - self.cen[0], x[1] - self.cen[1], x[2] - self.cen[2]
        M = self.metric(X, Y, Z)
        f, (k0, k1, k2) = M["f"], M["k"]
        # F^{jk} (h) from covariant b and contravariant d: al = b - f (d x k), h = (al + f k (k.al)) / (1 + f)
        al = (b[0] - f * (d[1] * k2 - d[2] * k1), b[1] - f * (d[2] * k0 - d[0] * k2), b[2] - f * (d[0] * k1 - d[1] * k0))
        ka = f * (k0 * al[0] + k1 * al[1] + k2 * al[2])
        inv = 1.0 / (1.0 + f)
        h = ((al[0] + ka * k0) * inv, (al[1] + ka * k1) * inv, (al[2] + ka * k2) * inv)
        # (q/m) F^{ac} u_c with u_c = g_cb u^b: u_i = u^i + f s k_i, u_4 = -u^4 + f s
        s = k0 * u[0] + k1 * u[1] + k2 * u[2] + u[3]
        fs = f * s
        c0, c1, c2 = u[0] + fs * k0, u[1] + fs * k1, u[2] + fs * k2
        c3 = fs - u[3]
        lor = (qm * (c1 * h[2] - c2 * h[1] + d[0] * c3), qm * (c2 * h[0] - c0 * h[2] + d[1] * c3),
               qm * (c0 * h[1] - c1 * h[0] + d[2] * c3), qm * (-(d[0] * c0 + d[1] * c1 + d[2] * c2)))
        gam = self.christoffel_uu(M, X, Y, Z, u)
        return [lor[q] - gam[q] for q in range(4)]

    # ---- Eq. 18 weights of one face ------------------------------------------------------------
    def integrand(self, pos, I, J):
        X, Y, Z = pos[0] - self.cen[0], pos[1] - self.cen[1], pos[2] - self.cen[2]
        M = self.metric(X, Y, Z)
        k = M["k"]
        return sqrt(1.0 + M["f"] * (k[I] * k[I] + k[J] * k[J]))

    def area(self, K, xK, I, Is, If, J, Js, Jf):
        ci, hi = 0.5 * (Is + If), 0.5 * (If - Is)
        cj, hj = 0.5 * (Js + Jf), 0.5 * (Jf - Js)
        s = None
        for p, wp in zip(self.gx, self.gw):
            for q, wq in zip(self.gx, self.gw):
                pos = [None, None, None]
                pos[K] = xK
                pos[I] = ci + hi * p
                pos[J] = cj + hj * q
                t = (wp * wq) * self.integrand(pos, I, J)
                s = t if s is None else s + t
        return s * 0.25 * (If - Is) * (Jf - Js)

    def deposit(self, x0, x1, qmacro, gbar, J):
        """Umeda's split of x0 -> x1 and the curved-metric face weights; adds to J[(K, node)]."""
        c1 = [int(math.floor(val(x0[ax]))) for ax in range(3)]
        c2 = [int(math.floor(val(x1[ax]))) for ax in range(3)]
        xr = []
        for ax in range(3):
            mid = 0.5 * (x0[ax] + x1[ax])
            lo, hi = float(min(c1[ax], c2[ax]) + 1), float(max(c1[ax], c2[ax]))
            xr.append(F(lo) if val(mid) > lo else (F(hi) if val(mid) < hi else mid))
        for seg, (a, b, cell) in enumerate(((x0, xr, c1), (xr, x1, c2))):
            P = [0.5 * (a[ax] + b[ax]) for ax in range(3)]
            for K in range(3):
                dK = b[K] - a[K]
                if val(dK) == 0.0:
                    continue
                flux = qmacro * gbar * dK / self.dt
                I, Jx = (K + 1) % 3, (K + 2) % 3
                i0, j0 = float(cell[I]), float(cell[Jx])
                A00 = self.area(K, P[K], I, P[I], i0 + 1.0, Jx, P[Jx], j0 + 1.0)
                A10 = self.area(K, P[K], I, F(i0), P[I], Jx, P[Jx], j0 + 1.0)
                A01 = self.area(K, P[K], I, P[I], i0 + 1.0, Jx, F(j0), P[Jx])
                A11 = self.area(K, P[K], I, F(i0), P[I], Jx, F(j0), P[Jx])
                FA = A00 + A10 + A01 + A11
                for (di, dj), A in zip(((0, 0), (1, 0), (0, 1), (1, 1)), (A00, A10, A01, A11)):
                    node = [0, 0, 0]
                    node[K], node[I], node[Jx] = cell[K], cell[I] + di, cell[Jx] + dj
                    key = (K, node[2], node[1], node[0])
                    J[key] = J.get(key, 0.0) + val(flux * (A / FA))

    # ---- one particle-step (Eqs. 13-16, deposit, removal) -----------------------------------
    def step(self, fields, x4, u4, qm, qmacro, gamma_in_j=True):
        """Returns (x1, u1, J contributions {(K, k, j, i): value}, removed)."""
        x0 = [F(v) for v in x4]
        u0 = [F(v) for v in u4]
        k1 = self.accel(fields, x0[:3], u0, qm)
        # Eq. 16: gamma_1 = [u^4/c + sqrt((u^4/c)^2 + 4 a^4 dt / (2c))] / 2
        w = u0[3] / self.c
        arg = w * w + 4.0 * k1[3] * (self.dt / (2.0 * self.c))
        g1 = 0.5 * (w + sqrt(arg)) if val(arg) >= 0.0 else w
        h = self.dt / g1
        sx, su = [], []
        xs = [x0[q] + (0.5 * h) * u0[q] for q in range(4)]
        us = [u0[q] + (0.5 * h) * k1[q] for q in range(4)]
        k2x, k2 = us, self.accel(fields, xs[:3], us, qm)
        xs = [x0[q] + (0.5 * h) * k2x[q] for q in range(4)]
        us = [u0[q] + (0.5 * h) * k2[q] for q in range(4)]
        k3x, k3 = us, self.accel(fields, xs[:3], us, qm)
        xs = [x0[q] + h * k3x[q] for q in range(4)]
        us = [u0[q] + h * k3[q] for q in range(4)]
        k4x, k4 = us, self.accel(fields, xs[:3], us, qm)
        h6 = h / 6.0
        x1 = [x0[q] + h6 * (u0[q] + 2.0 * k2x[q] + 2.0 * k3x[q] + k4x[q]) for q in range(4)]
        u1 = [u0[q] + h6 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]) for q in range(4)]
        del sx, su
        gbar = (u0[3] + u1[3]) / (2.0 * self.c) if gamma_in_j else F(1.0)
        J = {}
        if qmacro != 0.0:
            self.deposit(x0[:3], x1[:3], qmacro, gbar, J)
        # removal: r <= r_+ (the quartic at x_{n+1})
        X, Y, Z = x1[0] - self.cen[0], x1[1] - self.cen[1], x1[2] - self.cen[2]
        R2 = X * X + Y * Y + Z * Z
        p = R2 - self.a2
        q = self.a2 * (Z * Z)
        D = sqrt(p * p + 4.0 * q)
        r2 = 0.5 * (p + D) if val(p) >= 0.0 else (2.0 * q) / (D - p)
        removed = val(r2) <= self.r_plus ** 2
        return [val(v) for v in x1], [val(v) for v in u1], J, removed


def count_step(run, fields, x4, u4, qm, qmacro, gamma_in_j=True):
    """(operations, result) of one particle-step."""
    _C.n = 0
    res = run.step(fields, x4, u4, qm, qmacro, gamma_in_j)
    return _C.n, res
