// Fused gather + GR-RK4 push + curved-metric current deposit (Sec. 3.3 and Sec. 4).
//
// Per particle and step:
//   1. RK4 in proper time (Eqs. 13-16): y = (x^a, u^a), dy/dtau = (u, a~(x, u)),
//      a~ = (q/m) F^a_b u^b - Gamma^a_mn u^m u^n, one step h = dt / gamma_1 with gamma_1 from
//      Eq. 16 at (x_n, u_n); classical stage offsets 0, h/2, h/2, h.
//   2. At each stage: CIC gather of the six prognostic components, each from its own staggered
//      lattice (the sqrt(-det g) sub-volumes of Sec. 3.3 are exactly trilinear since
//      det g = -1), conversion with g at the particle, Lorentz + Christoffel terms.
//   3. Umeda zig-zag split of x_n -> x_{n+1} into two segments; the flux of each segment
//      through the faces of its cell, weighted by the four sub-areas of Eq. 18
//      (integrand sqrt(g_II g_JJ - g_IJ^2) = sqrt(1 + f (k_I^2 + k_J^2)), Q x Q Gauss-Legendre
//      per sub-rectangle, plane at the segment midpoint), times gamma_bar = (u^4_n+u^4_{n+1})/2c
//      (J = rho gamma v).
//   4. Removal flag: r <= r_+ or a coordinate outside [1, n-2]; sort key = cell or kDead.
//
// Precision: T = double runs everything in FP64.  T = float (FP32-mixed) keeps positions,
// velocities, fields and arithmetic in FP32 except where the FP32 estimate of r is below
// r_fp64 (default 4m): there the quartic, the metric and the Christoffel contraction are
// evaluated again in FP64.  The global J accumulators are FP64 in both modes.
//
// This GPU executes FP64 arithmetic, and conversions to and from FP64, at a small fraction of
// the FP32 rate on a pipe of its own.  So the FP32 path converts nothing per particle: the
// constants of a launch come in the arithmetic type (Consts), and the FP32 values added to
// the FP64 J accumulators are widened with integer operations (widen below).
#pragma once

#include <cmath>

#include "common.cuh"
#include "metric.cuh"

namespace grpic {

namespace {

template <int Q>
struct Gauss;
template <>
struct Gauss<1> {
  __device__ static constexpr double x(int) { return 0.0; }
  __device__ static constexpr double w(int) { return 2.0; }
};
template <>
struct Gauss<2> {
  __device__ static constexpr double x(int i) { return i == 0 ? -0.57735026918962576451 : 0.57735026918962576451; }
  __device__ static constexpr double w(int) { return 1.0; }
};
template <>
struct Gauss<3> {
  __device__ static constexpr double x(int i) {
    return i == 0 ? -0.77459666924148337704 : (i == 1 ? 0.0 : 0.77459666924148337704);
  }
  __device__ static constexpr double w(int i) { return i == 1 ? 8.0 / 9.0 : 5.0 / 9.0; }
};

// A block's shared-memory tile of J (FP32; three component planes of nx * ny * nz nodes starting
// at node (ox, oy, oz)), or tile == nullptr: deposits go straight to the global FP64 J.
struct JTile {
  float* tile = nullptr;
  int ox = 0, oy = 0, oz = 0;
  int nx = 0, ny = 0, nz = 0;
};


__device__ __forceinline__ double to_f64(float v) { return widen(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

template <typename T>
__device__ __forceinline__ T lerp(T a, T b, T w) {
  return fma(w, b - a, a);
}

template <typename T>
__device__ __forceinline__ T sel3(int i, T a, T b, T c) {
  return i == 0 ? a : (i == 1 ? b : c);
}

// FP64 r^2 at a grid position near the hole from the FP32 root s0 = r^2 (with the FP32
// D0 = sqrt((R^2 - a^2)^2 + 4 a^2 z^2)), by one Newton step on the quartic (Eq. 6).  With s = r^2
// it reads F(s) = s^2 - p s - q = 0 (p = R^2 - a^2, q = a^2 z^2); F'(s) = 2s - p = D at the root,
// and D >= s there (the difference of the two roots).  For s0 = s (1 + e) and D0 = D (1 + d),
// s0 - F(s0)/D0 has relative error about e (d - e s/D), i.e. ~1e-14: F(s0) is formed in FP64
// (it cancels), its quotient by D0 in FP32.  A poor FP32 start (a correction above 1e-5 s0,
// or s0 <= 0) takes the closed form in FP64.  X, Y, Z: the point minus the centre, in FP64.
__device__ __forceinline__ double quartic_newton(const Consts<float>& C, double X, double Y, double Z, float s0,
                                                 float D0, double* p_out) {
  const double p = fma(X, X, fma(Y, Y, fma(Z, Z, -C.da2)));
  *p_out = p;
  if (s0 > 0.f && D0 > 0.f) {
    const double q = C.da2 * Z * Z;
    const double S = widen(s0);
    const float corr = narrow(fma(S, S - p, -q)) / D0;
    if (fabsf(corr) <= 1e-5f * s0) return S - widen(corr);
  }
  double D;
  return kerr_r2<double, SeededOps64>(X, Y, Z, C.da, &D);
}

// FP64 metric and Christoffel contraction at a grid position (the FP32-mixed policy near the
// hole), from the FP32 r and D of the same point: r^2 by quartic_newton, D = 2 r^2 - p (the
// derivative of the quartic at its root), reciprocals and roots by SeededOps64; f, k and the
// contraction in FP64, rounded to FP32.  Out of line: it runs for few particles.
__device__ __noinline__ void metric_christoffel_fp64(const Consts<float>& C, float x, float y, float z, float u0,
                                                     float u1, float u2, float u3, float rf, float Df, float* out) {
  const double Xd = widen(x) - C.dxc, Yd = widen(y) - C.dyc, Zd = widen(z) - C.dzc;
  double p;
  const double s = quartic_newton(C, Xd, Yd, Zd, rf * rf, Df, &p);
  const Kerr<double> K = kerr_from_r2<double, SeededOps64>(Xd, Yd, Zd, C.dm, C.da, s, 2.0 * s - p);
  const double ud[4] = {widen(u0), widen(u1), widen(u2), widen(u3)};
  double gd[4];
  christoffel_uu<double, SeededOps64>(K, Xd, Yd, Zd, C.da, ud, gd);
  out[0] = narrow(K.f);
  out[1] = narrow(K.k0);
  out[2] = narrow(K.k1);
  out[3] = narrow(K.k2);
  out[4] = narrow(gd[0]);
  out[5] = narrow(gd[1]);
  out[6] = narrow(gd[2]);
  out[7] = narrow(gd[3]);
}

// FP64 root of the quartic (Eq. 6) at a quadrature node near the hole (absolute FP32 node
// coordinates px, py, pz), as r^2 rounded to FP32.
__device__ __noinline__ float quartic_fp64(const Consts<float>& C, float px, float py, float pz, float s0,
                                           float D0) {
  double p;
  return narrow(quartic_newton(C, widen(px) - C.dxc, widen(py) - C.dyc, widen(pz) - C.dzc, s0, D0, &p));
}

// a~ at (x, u): gather, convert, Lorentz - Christoffel.
// mixed: the FP32-mixed policy applies (T = float): where the FP32 r is below r_fp64 the metric
// and the Christoffel contraction are taken from metric_christoffel_fp64.
template <typename T>
__device__ __forceinline__ void accel(const Grid& g, const Fields<T>& F, const Consts<T>& C, const T x[3],
                                      const T u[4], T out[4], unsigned& flags, unsigned& n64, bool mixed) {
  // --- CIC gather: integer lattice (floor x) and half lattice (floor(x - 1/2)) per axis
  int ii[3], ih[3];
  T wi[3], wh[3];
  const int nn[3] = {g.nx, g.ny, g.nz};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const T s0 = x[ax];
    const T s1 = x[ax] - T(0.5);
    if (!(s1 >= T(0)) || !(s0 <= T(nn[ax] - 1))) flags |= ST_RANGE;
    int a0 = (int)floor(s0), a1 = (int)floor(s1);
    a0 = min(max(a0, 0), nn[ax] - 2);
    a1 = min(max(a1, 0), nn[ax] - 2);
    ii[ax] = a0;
    ih[ax] = a1;
    wi[ax] = s0 - T(a0);
    wh[ax] = s1 - T(a1);
  }
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  T val[6];
#pragma unroll
  for (int comp = 0; comp < 6; ++comp) {
    // lattice offsets: d^x (1,0,0) d^y (0,1,0) d^z (0,0,1) b_x (0,1,1) b_y (1,0,1) b_z (1,1,0)
    const bool hx = (comp == 0) || (comp == 4) || (comp == 5);
    const bool hy = (comp == 1) || (comp == 3) || (comp == 5);
    const bool hz = (comp == 2) || (comp == 3) || (comp == 4);
    const int i0 = hx ? ih[0] : ii[0], j0 = hy ? ih[1] : ii[1], k0 = hz ? ih[2] : ii[2];
    const T w0 = hx ? wh[0] : wi[0], w1 = hy ? wh[1] : wi[1], w2 = hz ? wh[2] : wi[2];
    const T* arr = comp < 3 ? F.d[comp] : F.b[comp - 3];
    const T* q = arr + (((long long)k0 * g.ny + j0) * g.nx + i0);
    // trilinear as nested linear interpolations (the weight products expanded, 7 lerps)
    const T c00 = lerp(__ldg(q), __ldg(q + 1), w0);
    const T c10 = lerp(__ldg(q + sy), __ldg(q + sy + 1), w0);
    const T c01 = lerp(__ldg(q + sz), __ldg(q + sz + 1), w0);
    const T c11 = lerp(__ldg(q + sz + sy), __ldg(q + sz + sy + 1), w0);
    val[comp] = lerp(lerp(c00, c10, w1), lerp(c01, c11, w1), w2);
  }
  const T d[3] = {val[0], val[1], val[2]};
  const T b[3] = {val[3], val[4], val[5]};

  // --- metric and Christoffel contraction at the particle
  T f, k0, k1, k2, gam[4];
  const T X = x[0] - C.xc, Y = x[1] - C.yc, Z = x[2] - C.zc;
  const Kerr<T> Kt = kerr_eval<T>(X, Y, Z, C.m, C.a);
  bool promoted = false;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (mixed && Kt.r < C.r_fp64) {
      float o[8];
      metric_christoffel_fp64(C, x[0], x[1], x[2], u[0], u[1], u[2], u[3], Kt.r, Kt.D, o);
      f = o[0];
      k0 = o[1];
      k1 = o[2];
      k2 = o[3];
      gam[0] = o[4];
      gam[1] = o[5];
      gam[2] = o[6];
      gam[3] = o[7];
      ++n64;
      promoted = true;
    }
  }
  if (!promoted) {
    christoffel_uu<T>(Kt, X, Y, Z, C.a, u, gam);
    f = Kt.f;
    k0 = Kt.k0;
    k1 = Kt.k1;
    k2 = Kt.k2;
  }
  T h[3], lor[4];
  contra_spatial(f, k0, k1, k2, b, d, h);
  lorentz(C.qm, f, k0, k1, k2, h, d, u, lor);
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = lor[q] - gam[q];
}

// Integrand of Eq. 18, sqrt(g_II g_JJ - g_IJ^2) = sqrt(1 + f (k_I^2 + k_J^2)), at a grid
// position (the FP64 path; the FP32 paths use deposit_lattice).
template <typename T>
__device__ __forceinline__ T area_integrand(const Consts<T>& C, T px, T py, T pz, int K) {
  const T X = px - C.xc, Y = py - C.yc, Z = pz - C.zc;
  T D;
  const T r2 = kerr_r2<T>(X, Y, Z, C.a, &D);
  return area_density<T>(X, Y, Z, C.m, C.a, r2, K);
}

// AREA of Eq. 18 over [Is, If] x [Js, Jf] in the plane x^K = xK.
template <typename T, int Q>
__device__ __forceinline__ T area(const Consts<T>& C, int K, T xK, T Is, T If, T Js, T Jf) {
  T s = T(0);
  const T ci = T(0.5) * (Is + If), hi = T(0.5) * (If - Is);
  const T cj = T(0.5) * (Js + Jf), hj = T(0.5) * (Jf - Js);
#pragma unroll
  for (int p = 0; p < Q; ++p)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T xi = ci + hi * (T)Gauss<Q>::x(p);
      const T xj = cj + hj * (T)Gauss<Q>::x(q);
      // (x^K, x^I, x^J) -> (x, y, z) with I = K+1, J = K+2 (mod 3)
      const T px = sel3(K, xK, xj, xi);
      const T py = sel3(K, xi, xK, xj);
      const T pz = sel3(K, xj, xi, xK);
      s += (T)Gauss<Q>::w(p) * (T)Gauss<Q>::w(q) * area_integrand<T>(C, px, py, pz, K);
    }
  return s * T(0.25) * (If - Is) * (Jf - Js);
}

// Umeda zig-zag deposit of the move x0 -> x0 + dx.  The segment displacements are carried
// as offsets from x0 (s1 = relay - x0, s2 = dx - s1), so the flux keeps the accuracy of the RK4
// increment instead of inheriting the rounding of the stored positions.  With |dx| < 1 the
// relay point min(min(a,b)+1, max(max(a,b), mid)) is the midpoint when the cell does not
// change along an axis and the shared face otherwise.
template <typename T, int Q>
__device__ __forceinline__ void deposit(const Grid& g, const Fields<T>& F, const Consts<T>& C, const T x0[3],
                                        const T dx[3], T qg, T inv_dt, unsigned& flags) {
  const int nn[3] = {g.nx, g.ny, g.nz};
  int c1[3], c2[3];
  T s1[3], s2[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    int a = (int)floor(x0[ax]), b = (int)floor(x0[ax] + dx[ax]);
    if (a < 0 || b < 0 || a > nn[ax] - 2 || b > nn[ax] - 2) flags |= ST_RANGE;
    a = min(max(a, 0), nn[ax] - 2);
    b = min(max(b, 0), nn[ax] - 2);
    c1[ax] = a;
    c2[ax] = b;
    s1[ax] = (a == b) ? T(0.5) * dx[ax] : (T)max(a, b) - x0[ax];
    s2[ax] = dx[ax] - s1[ax];
  }
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
#pragma unroll 1
  for (int seg = 0; seg < 2; ++seg) {
    const int cx = seg ? c2[0] : c1[0], cy = seg ? c2[1] : c1[1], cz = seg ? c2[2] : c1[2];
    T P[3], dseg[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      dseg[ax] = seg ? s2[ax] : s1[ax];
      P[ax] = seg ? x0[ax] + (s1[ax] + T(0.5) * s2[ax]) : x0[ax] + T(0.5) * s1[ax];
    }
    const long long base = ((long long)cz * g.ny + cy) * g.nx + cx;
#pragma unroll 1
    for (int K = 0; K < 3; ++K) {
      const T dK = sel3(K, dseg[0], dseg[1], dseg[2]);
      if (dK == T(0)) continue;
      const T flux = qg * dK * inv_dt;
      const T PK = sel3(K, P[0], P[1], P[2]);
      const T PI = sel3(K, P[1], P[2], P[0]);
      const T PJ = sel3(K, P[2], P[0], P[1]);
      const T i0 = (T)sel3(K, cy, cz, cx), j0 = (T)sel3(K, cz, cx, cy);
      const T A00 = area<T, Q>(C, K, PK, PI, i0 + T(1), PJ, j0 + T(1));
      const T A10 = area<T, Q>(C, K, PK, i0, PI, PJ, j0 + T(1));
      const T A01 = area<T, Q>(C, K, PK, PI, i0 + T(1), j0, PJ);
      const T A11 = area<T, Q>(C, K, PK, i0, PI, j0, PJ);
      const T FA = A00 + A10 + A01 + A11;
      const T W00 = A00 / FA, W10 = A10 / FA, W01 = A01 / FA, W11 = A11 / FA;
      const long long stI = sel3(K, sy, sz, 1ll), stJ = sel3(K, sz, 1ll, sy);
      double* JK = sel3(K, F.J[0], F.J[1], F.J[2]);
      atomicAdd(JK + base, to_f64(flux * W00));
      atomicAdd(JK + base + stI, to_f64(flux * W10));
      atomicAdd(JK + base + stJ, to_f64(flux * W01));
      atomicAdd(JK + base + stI + stJ, to_f64(flux * W11));
    }
  }
}

// A quadrature node that the far-field formula of deposit_lattice does not cover (FP32-mixed
// warps only): the p <= 0 branch of the quartic (the cancellation-free form), and the FP64
// policy where the FP32 r is below r_fp64 (or always, with promote).  Returns r^2 and whether
// it came from FP64.  Out of line: far-field warps never call it.
__device__ __noinline__ float2 node_slow(const Consts<float>& C, float p, float q, float ax, float ay, float az,
                                         bool promote) {
  const float D = sqrtf(fmaf(p, p, 4.f * q));
  float r2 = p >= 0.f ? 0.5f * (p + D) : __fdividef(2.f * q, D - p);
  if (promote || !(r2 >= C.r2_fp64)) return make_float2(quartic_fp64(C, ax, ay, az, r2, D), 1.f);
  return make_float2(r2, 0.f);
}

// FP32 deposit (the zig-zag split, fluxes and Eq. 18 weights of deposit() below) evaluated on a
// per-face node lattice: the Q x Q Gauss nodes of the four sub-rectangles of a face make a
// 2Q x 2Q lattice in (x^I, x^J), so node coordinates, their squares and the spin terms are
// formed once per face, roots are v * rsqrt(v) and each node needs one reciprocal.
//   Integrand: 1 + f (1 - k_K^2) with f = 2 m r^3 / Sigma, Sigma = r^4 + a^2 z^2, and
//   1 - k_z^2 = (r^2 - z^2) / r^2;  1 - k_x^2 = (rho^4 - (r x - a y)^2) / rho^4,
//   1 - k_y^2 = (rho^4 - (r y + a x)^2) / rho^4,  rho^2 = r^2 + a^2.
// With (I, J) = (K+1, K+2) mod 3: K = 0 -> (x, y, z) = (x^K, x^I, x^J); K = 1 -> (x^J, x^K, x^I);
// K = 2 -> (x^I, x^J, x^K).
// Every node first takes the far-field form: for a particle outside the near radius every node
// has R > |a|, so the quartic takes its p = R^2 - a^2 > 0 branch and every root argument is
// positive.  With mixed (a warp-uniform flag) a node with p <= 0 or an FP32 r below r_fp64 is
// handed to node_slow (the FP64 policy, quartic_fp64 at the node's FP32 coordinates), and r = 0
// gives the flat limit; one code path serves far-field and mixed warps alike.
template <int Q>
__device__ __forceinline__ void deposit_lattice(const Grid& g, const Fields<float>& F, const Consts<float>& C,
                                                const float x0[3], const float dx[3], float qg, float inv_dt,
                                                unsigned& flags, unsigned& n64, bool mixed, const JTile& jt) {
  const int nn[3] = {g.nx, g.ny, g.nz};
  int c1[3], c2[3];
  float s1[3], s2[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    int a = (int)floorf(x0[ax]), b = (int)floorf(x0[ax] + dx[ax]);
    if (a < 0 || b < 0 || a > nn[ax] - 2 || b > nn[ax] - 2) flags |= ST_RANGE;
    a = min(max(a, 0), nn[ax] - 2);
    b = min(max(b, 0), nn[ax] - 2);
    c1[ax] = a;
    c2[ax] = b;
    s1[ax] = (a == b) ? 0.5f * dx[ax] : (float)max(a, b) - x0[ax];
    s2[ax] = dx[ax] - s1[ax];
  }
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  const float cen[3] = {C.xc, C.yc, C.zc};
#pragma unroll 1
  for (int seg = 0; seg < 2; ++seg) {
    const int cx = seg ? c2[0] : c1[0], cy = seg ? c2[1] : c1[1], cz = seg ? c2[2] : c1[2];
    float P[3], dseg[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      dseg[ax] = seg ? s2[ax] : s1[ax];
      P[ax] = seg ? x0[ax] + (s1[ax] + 0.5f * s2[ax]) : x0[ax] + 0.5f * s1[ax];
    }
    const long long base = ((long long)cz * g.ny + cy) * g.nx + cx;
#pragma unroll 1
    for (int K = 0; K < 3; ++K) {
      const float dK = sel3(K, dseg[0], dseg[1], dseg[2]);
      if (dK == 0.f) continue;
      const float flux = qg * dK * inv_dt;
      const float PK = sel3(K, P[0], P[1], P[2]);
      const float XK = PK - sel3(K, cen[0], cen[1], cen[2]);
      const float PI = sel3(K, P[1], P[2], P[0]), PJ = sel3(K, P[2], P[0], P[1]);
      const float i0 = (float)sel3(K, cy, cz, cx), j0 = (float)sel3(K, cz, cx, cy);
      const float cI = sel3(K, cen[1], cen[2], cen[0]), cJ = sel3(K, cen[2], cen[0], cen[1]);
      // node lattice: sub-interval 0 = [i0, PI], 1 = [PI, i0 + 1] (likewise in J); AJ the nodes'
      // grid coordinates along J, XJ relative to the centre.  The rows (along I) run in a rolled
      // loop, the nodes of a row unrolled: a quarter of the code of a fully unrolled lattice, so
      // the far-field and FP32-mixed copies of a kernel fit the instruction cache together.
      const float wI0 = PI - i0, wI1 = i0 + 1.f - PI;
      // Per node the quartic needs p = R^2 - a^2 and q = a^2 z^2, k_K's numerator the spin term
      // -a x^I (K = 0) or +a x^J (K = 1); z is x^K, x^I or x^J (K = 2, 1, 0).  Each of these is a
      // sum of a face constant, a row term and a column term, formed once: a node adds them.
      const float pK = XK * XK - C.a2;
      const float qK = K == 2 ? C.a2 * XK * XK : 0.f;
      float AJ[2 * Q], XJ[2 * Q], pJ[2 * Q], qJ[2 * Q], tJ[2 * Q], wJ[2];
#pragma unroll
      for (int sub = 0; sub < 2; ++sub) {
        const float lo_j = sub ? PJ : j0, hi_j = sub ? j0 + 1.f : PJ;
        wJ[sub] = hi_j - lo_j;
#pragma unroll
        for (int p = 0; p < Q; ++p) {
          const int jb = sub * Q + p;
          AJ[jb] = 0.5f * (lo_j + hi_j) + 0.5f * wJ[sub] * (float)Gauss<Q>::x(p);
          XJ[jb] = AJ[jb] - cJ;
          pJ[jb] = XJ[jb] * XJ[jb];
          qJ[jb] = K == 0 ? C.a2 * pJ[jb] : 0.f;
          tJ[jb] = K == 1 ? C.a * XJ[jb] : 0.f;
        }
      }
      float S00 = 0.f, S01 = 0.f, S10 = 0.f, S11 = 0.f;  // S[sub I][sub J]
#pragma unroll 1
      for (int ia = 0; ia < 2 * Q; ++ia) {
        const int si = ia >= Q ? 1 : 0, pi = ia - si * Q;
        float gx = (float)Gauss<Q>::x(0), gw = (float)Gauss<Q>::w(0);
#pragma unroll
        for (int t = 1; t < Q; ++t)
          if (pi == t) {
            gx = (float)Gauss<Q>::x(t);
            gw = (float)Gauss<Q>::w(t);
          }
        const float lo_i = si ? PI : i0, w_i = si ? wI1 : wI0;
        const float AIa = lo_i + 0.5f * w_i + 0.5f * w_i * gx;
        const float XIa = AIa - cI;
        const float XI2 = XIa * XIa;
        const float pRow = pK + XI2;
        const float qRow = qK + (K == 1 ? C.a2 * XI2 : 0.f);
        const float tRow = K == 0 ? -C.a * XIa : 0.f;
        float row0 = 0.f, row1 = 0.f;
#pragma unroll
        for (int jb = 0; jb < 2 * Q; ++jb) {
          const float p = pRow + pJ[jb];
          const float q = qRow + qJ[jb];
          const float D2 = fmaf(p, p, 4.f * q);
          float r2 = 0.5f * (p + D2 * rsqrtf(D2));
          float val;
          if (mixed && (!(p > 0.f) || !(r2 >= C.r2_fp64))) {
            const float ax = sel3(K, PK, AJ[jb], AIa), ay = sel3(K, AIa, PK, AJ[jb]);
            const float az = sel3(K, AJ[jb], AIa, PK);
            const float2 rs = node_slow(C, p, q, ax, ay, az, p > 0.f);
            r2 = rs.x;
            n64 += (unsigned)rs.y;
          }
          if (mixed && !(r2 > 0.f)) {
            val = 1.f;  // the flat limit r = 0
          } else {
            const float r = r2 * rsqrtf(r2);
            const float sig = fmaf(r2, r2, q);
            float fperp;
            if (K == 2) {
              fperp = __fdividef(C.two_m * r * (r2 - XK * XK), sig);
            } else {
              const float num = fmaf(r, XK, tRow + tJ[jb]);
              const float rho2 = r2 + C.a2;
              const float rho4 = rho2 * rho2;
              fperp = __fdividef(C.two_m * r * r2 * fmaf(-num, num, rho4), rho4 * sig);
            }
            const float v = 1.f + fperp;
            val = v * rsqrtf(v);
          }
          if (jb < Q)
            row0 += (float)Gauss<Q>::w(jb % Q) * val;
          else
            row1 += (float)Gauss<Q>::w(jb % Q) * val;
        }
        if (si == 0) {
          S00 += gw * row0;
          S01 += gw * row1;
        } else {
          S10 += gw * row0;
          S11 += gw * row1;
        }
      }
      const float wI[2] = {wI0, wI1};
      const float S[2][2] = {{S00, S01}, {S10, S11}};
      // sub-rectangle areas; a node's weight is the area of the sub-rectangle opposite it
      const float A00 = S[1][1] * 0.25f * wI[1] * wJ[1];
      const float A10 = S[0][1] * 0.25f * wI[0] * wJ[1];
      const float A01 = S[1][0] * 0.25f * wI[1] * wJ[0];
      const float A11 = S[0][0] * 0.25f * wI[0] * wJ[0];
      const float rFA = __fdividef(1.f, A00 + A10 + A01 + A11);
      // the face's four nodes: into the block's J tile when they lie in it, else into global J
      const int tx = cx - jt.ox, ty = cy - jt.oy, tz = cz - jt.oz;
      if (jt.tile && (unsigned)tx < (unsigned)(jt.nx - 1) && (unsigned)ty < (unsigned)(jt.ny - 1) &&
          (unsigned)tz < (unsigned)(jt.nz - 1)) {
        const int tsy = jt.nx, tsz = jt.nx * jt.ny;
        const int tI = sel3(K, tsy, tsz, 1), tJ = sel3(K, tsz, 1, tsy);
        float* TK = jt.tile + K * tsz * jt.nz + (tz * jt.ny + ty) * jt.nx + tx;
        atomicAdd(TK, flux * (A00 * rFA));
        atomicAdd(TK + tI, flux * (A10 * rFA));
        atomicAdd(TK + tJ, flux * (A01 * rFA));
        atomicAdd(TK + tI + tJ, flux * (A11 * rFA));
      } else {
        const long long stI = sel3(K, sy, sz, 1ll), stJ = sel3(K, sz, 1ll, sy);
        double* JK = sel3(K, F.J[0], F.J[1], F.J[2]);
        atomicAdd(JK + base, widen(flux * (A00 * rFA)));
        atomicAdd(JK + base + stI, widen(flux * (A10 * rFA)));
        atomicAdd(JK + base + stJ, widen(flux * (A01 * rFA)));
        atomicAdd(JK + base + stI + stJ, widen(flux * (A11 * rFA)));
      }
    }
  }
}

// One particle-step of particle i: RK4 push, deposit, removal flag and sort key (written to
// *key_out: P.key + i, or a side array where another kernel still reads P.key concurrently).
// mixed (T = float): the FP32-mixed policy applies to this warp's particles (a warp-uniform
// flag; false only where every particle lies outside near_radius).  T = double ignores it.
template <typename T, int Q>
__device__ __forceinline__ void push_particle(const Grid& g, const Fields<T>& F, const Particles<T>& P,
                                              const Consts<T>& C, long long i, DevStatus* st, unsigned& flags,
                                              unsigned& n64, uint32_t* key_out, bool mixed,
                                              const JTile& jt = JTile()) {
  T x0[4], u0[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    x0[q] = P.x[q][i];
    u0[q] = P.u[q][i];
  }
  // RK4 in proper time: stages at offsets 0, h/2, h/2, h; h = dt / gamma_1 (Eq. 16)
  T xs[4], us[4], a[4], sx[4], su[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    xs[q] = x0[q];
    us[q] = u0[q];
    sx[q] = T(0);
    su[q] = T(0);
  }
  T h = T(0);
  bool fb = false;
#pragma unroll 1
  for (int stage = 0; stage < 4; ++stage) {
    accel<T>(g, F, C, xs, us, a, flags, n64, mixed);
    if (stage == 0) h = C.dt / gamma_step<T>(u0[3], a[3], C.inv_c, C.dt, &fb);
    const T wgt = (stage == 0 || stage == 3) ? T(1) : T(2);
    const T frac = (stage == 2) ? h : T(0.5) * h;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sx[q] += wgt * us[q];
      su[q] += wgt * a[q];
      xs[q] = x0[q] + frac * us[q];
      us[q] = u0[q] + frac * a[q];
    }
  }
  T x1[4], u1[4], dx[4];
  const T h6 = h / T(6);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    dx[q] = h6 * sx[q];
    x1[q] = x0[q] + dx[q];
    u1[q] = u0[q] + h6 * su[q];
  }
  x1[3] -= C.cdt;  // x^4 is stored relative to c t
  bool finite = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) finite = finite && isfinite(x1[q]) && isfinite(u1[q]);
  if (!finite) flags |= ST_NONFINITE;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (!(fabs(x1[q] - x0[q]) < T(1))) flags |= ST_CFL;
  // deposit, J = rho gamma v
  if (finite && C.qmacro != T(0)) {
    const T gbar = C.gamma_in_j ? (u0[3] + u1[3]) / (T(2) * C.c) : T(1);
    if constexpr (sizeof(T) == sizeof(float))
      deposit_lattice<Q>(g, F, C, x0, dx, C.qmacro * gbar, C.inv_dt, flags, n64, mixed, jt);
    else
      deposit<T, Q>(g, F, C, x0, dx, C.qmacro * gbar, C.inv_dt, flags);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    P.x[q][i] = x1[q];
    P.u[q][i] = u1[q];
  }
  // removal (r <= r_+ or outside [1, n-2]) and the sort key
  bool outer = !finite;
  const int nn[3] = {g.nx, g.ny, g.nz};
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (!(x1[q] >= T(1) && x1[q] <= T(nn[q] - 2))) outer = true;
  bool horizon = false;
  if (finite && C.massive) {
    // screen in T, decide in FP64 near r_+
    const T X = x1[0] - C.xc, Y = x1[1] - C.yc, Z = x1[2] - C.zc;
    T D;
    const T r2 = kerr_r2<T>(X, Y, Z, C.a, &D);
    if (r2 < C.rcheck2) {
      double Dd;
      const double r2d =
          kerr_r2<double>(to_f64(x1[0]) - C.dxc, to_f64(x1[1]) - C.dyc, to_f64(x1[2]) - C.dzc, C.da, &Dd);
      horizon = !(r2d > 0.0) || sqrt(r2d) <= C.r_plus;
    }
  }
  if (horizon || outer) {
    *key_out = kDead;
    atomicAdd(horizon ? &st->removed_horizon : &st->removed_outer, 1ull);
  } else {
    const int ci = (int)floor(x1[0]), cj = (int)floor(x1[1]), ck = (int)floor(x1[2]);
    *key_out = (uint32_t)(((long long)ck * g.ny + cj) * g.nx + ci);
  }
  if (fb) atomicAdd(&st->fallbacks, 1ull);
}

// Warp-aggregated status: flags, FP64 evaluations and particle-steps of the warp's lanes.
__device__ __forceinline__ void warp_status(DevStatus* st, unsigned flags, unsigned n64, bool active) {
  const unsigned any_flags = __reduce_or_sync(0xffffffffu, flags);
  const unsigned sum64 = __reduce_add_sync(0xffffffffu, n64);
  const unsigned npush = __popc(__ballot_sync(0xffffffffu, active));
  if ((threadIdx.x & 31) == 0) {
    if (any_flags) atomicOr(&st->flags, any_flags);
    if (sum64) atomicAdd(&st->fp64_evals, (unsigned long long)sum64);
    if (npush) atomicAdd(&st->pushed, (unsigned long long)npush);
  }
}

}  // namespace

}  // namespace grpic
