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

#include <cuda_fp16.h>

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

// Packed FP32 pairs: one instruction performs the operation on both lanes, each lane rounded as
// the scalar operation would be.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }

// f and k of Eqs. 4-5 for a point whose quartic (Eq. 6) takes its p = R^2 - a^2 > 0 branch and
// r > 0 (every stage of a far-field particle, R > |a|): with h = p / 2, r^2 = h + sqrt(h^2 + q)
// and D = 2 sqrt(h^2 + q); the reciprocal square roots give 1/D and 1/r as well, and since the
// root satisfies Sigma = r^4 + a^2 z^2 = r^2 D, 1/Sigma and f = 2 m r / D need no division.
__device__ __forceinline__ Kerr<float> kerr_far(float x, float y, float z, float m, float a) {
  Kerr<float> K;
  const float a2 = a * a;
  const float q = a2 * z * z;
  const float h = 0.5f * (x * x + y * y + z * z - a2);
  const float Dh2 = fmaf(h, h, q);
  const float rDh = rsqrtf(Dh2);
  const float r2 = fmaf(Dh2, rDh, h);
  K.flat = false;
  K.D = 2.f * Dh2 * rDh;
  K.inv_D = 0.5f * rDh;
  K.inv_r = rsqrtf(r2);
  K.r = r2 * K.inv_r;
  K.inv_rho2 = __fdividef(1.f, r2 + a2);
  K.inv_sig = K.inv_D * K.inv_r * K.inv_r;
  K.f = m * K.r * rDh;
  K.k0 = (K.r * x - a * y) * K.inv_rho2;
  K.k1 = (K.r * y + a * x) * K.inv_rho2;
  K.k2 = z * K.inv_r;
  return K;
}

// Gamma^a_mn u^m u^n of christoffel_uu (metric.cuh) in FP32, the x and y components of its
// 3-vectors, and of each row of the Jacobian d_i k_j, as packed pairs.
__device__ __forceinline__ void christoffel_uu_x2(const Kerr<float>& K, float x, float y, float z, float a,
                                                  const float u[4], float out[4]) {
  if (K.flat) {
    out[0] = out[1] = out[2] = out[3] = 0.f;
    return;
  }
  const float r = K.r, f = K.f, k2 = K.k2;
  const float2 kxy = make_float2(K.k0, K.k1), xy = make_float2(x, y);
  const float r2 = r * r, a2 = a * a;
  const float inv_rho2 = K.inv_rho2, inv_D = K.inv_D, inv_r = K.inv_r, inv_sig = K.inv_sig;
  // grad r (r_x, r_y) = (x, y) r / D, r_z = z (r^2 + a^2) / (r D); grad f as in christoffel_uu
  const float2 rxy = mul2(xy, f2(r * inv_D));
  const float rz = z * (r2 + a2) * inv_D * inv_r;
  const float fr = f * (3.f * inv_r - 4.f * r2 * r * inv_sig);
  const float2 fxy = mul2(f2(fr), rxy);
  const float fz = fr * rz - 2.f * a2 * z * f * inv_sig;
  // row i of J[i][j] = d_i k_j: (J[i][0], J[i][1]) packed, J[i][2] alone
  const float ri[3] = {rxy.x, rxy.y, rz};
  float2 J01[3];
  float J2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float tr = 2.f * r * ri[i];
    const float2 c = i == 0 ? make_float2(r, a) : (i == 1 ? make_float2(-a, r) : make_float2(0.f, 0.f));
    J01[i] = mul2(fma2(f2(-tr), kxy, fma2(xy, f2(ri[i]), c)), f2(inv_rho2));
    J2[i] = ((i == 2 ? 1.f : 0.f) - k2 * ri[i]) * inv_r;
  }
  const float s = K.k0 * u[0] + K.k1 * u[1] + k2 * u[2] + u[3];
  const float2 ufxy = mul2(make_float2(u[0], u[1]), fxy);
  const float uf = ufxy.x + ufxy.y + u[2] * fz;
  // D_j = u^i J[i][j], E_j = u^i J[j][i]
  const float2 D01 = fma2(f2(u[0]), J01[0], fma2(f2(u[1]), J01[1], mul2(f2(u[2]), J01[2])));
  const float D2 = u[0] * J2[0] + u[1] * J2[1] + u[2] * J2[2];
  float E[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) E[j] = u[0] * J01[j].x + u[1] * J01[j].y + u[2] * J2[j];
  const float uD = u[0] * D01.x + u[1] * D01.y + u[2] * D2;
  const float c1 = uf * s + f * uD;
  const float fs = f * s;
  const float hs2 = 0.5f * s * s;
  const float2 w01 =
      fma2(f2(c1), kxy, fma2(f2(fs), D01, fma2(f2(-fs), make_float2(E[0], E[1]), mul2(f2(-hs2), fxy))));
  const float w2 = c1 * k2 + fs * (D2 - E[2]) - hs2 * fz;
  const float kw = K.k0 * w01.x + K.k1 * w01.y + k2 * w2 - c1;
  const float2 o01 = fma2(f2(-f * kw), kxy, w01);
  out[0] = o01.x;
  out[1] = o01.y;
  out[2] = w2 - f * k2 * kw;
  out[3] = -c1 + f * kw;
}

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

// The non-negative root of Eq. 6 as r^2 in FP64 from p = R^2 - a^2 and q = a^2 z^2 (the
// cancellation-free branch form), for a quadrature node whose Newton start was poor.
__device__ __noinline__ double quartic_closed64(double p, double q) {
  const double D = SeededOps64::root(fma(p, p, 4.0 * q));
  return p >= 0.0 ? 0.5 * (p + D) : SeededOps64::div(2.0 * q, D - p);
}

// FP64 r^2 of a quadrature node from its FP64 p and q, by the Newton step of quartic_newton from
// the FP32 root s0 (FP32 D0), rounded to FP32.  With |corr| <= 1e-5 s0 the difference s0 - corr of
// two FP32 numbers is exact in FP64, so its rounding to FP32 is the FP32 subtraction itself.
__device__ __forceinline__ float node_newton64(double p, double q, float s0, float D0) {
  if (s0 > 0.f && D0 > 0.f) {
    const double S = widen(s0);
    const float corr = narrow(fma(S, S - p, -q)) / D0;
    if (fabsf(corr) <= 1e-5f * s0) return s0 - corr;
  }
  return narrow(quartic_closed64(p, q));
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
    if constexpr (sizeof(T) == sizeof(float)) {
      // the lerps along x of the (z0, z1) pairs at y0 and at y1, then along y, as packed pairs;
      // b - a = fma(a, -1, b) exactly, so each lane equals the scalar lerp
      const float2 a0 = make_float2(__ldg(q), __ldg(q + sz)), a1 = make_float2(__ldg(q + 1), __ldg(q + sz + 1));
      const float2 b0 = make_float2(__ldg(q + sy), __ldg(q + sz + sy));
      const float2 b1 = make_float2(__ldg(q + sy + 1), __ldg(q + sz + sy + 1));
      const float2 cy0 = fma2(f2(w0), fma2(a0, f2(-1.f), a1), a0);
      const float2 cy1 = fma2(f2(w0), fma2(b0, f2(-1.f), b1), b0);
      const float2 cz = fma2(f2(w1), fma2(cy0, f2(-1.f), cy1), cy0);
      val[comp] = lerp(cz.x, cz.y, w2);
    } else {
      const T c00 = lerp(__ldg(q), __ldg(q + 1), w0);
      const T c10 = lerp(__ldg(q + sy), __ldg(q + sy + 1), w0);
      const T c01 = lerp(__ldg(q + sz), __ldg(q + sz + 1), w0);
      const T c11 = lerp(__ldg(q + sz + sy), __ldg(q + sz + sy + 1), w0);
      val[comp] = lerp(lerp(c00, c10, w1), lerp(c01, c11, w1), w2);
    }
  }
  const T d[3] = {val[0], val[1], val[2]};
  const T b[3] = {val[3], val[4], val[5]};

  // --- metric and Christoffel contraction at the particle
  T f, k0, k1, k2, gam[4];
  const T X = x[0] - C.xc, Y = x[1] - C.yc, Z = x[2] - C.zc;
  Kerr<T> Kt;
  if constexpr (sizeof(T) == sizeof(float)) {
    // far-field warps: every stage has R > |a| (the quartic's p > 0 branch)
    Kt = mixed ? kerr_eval<T>(X, Y, Z, C.m, C.a) : kerr_far(X, Y, Z, C.m, C.a);
  } else {
    Kt = kerr_eval<T>(X, Y, Z, C.m, C.a);
  }
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
    if constexpr (sizeof(T) == sizeof(float))
      christoffel_uu_x2(Kt, X, Y, Z, C.a, u, gam);
    else
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

// The per-face quantities of deposit_lattice and the per-node terms they are built from (one
// definition, so that the deferred near-hole nodes see exactly the values of the main loop).
struct FaceLattice {
  int K;
  float PK, XK, PI, PJ, i0, j0, cI, cJ, wI0, wI1, pK, qK;
  // factors of the row and column terms of q = a^2 z^2 and of the spin term of k_K's numerator
  // (a^2, -a, a or 0 by K), so that every term is a product instead of a choice
  float qI, tI, qJ, tJ;
};

// Grid coordinate along I of lattice row ia = si * Q + pi, and the row terms of p, q and the
// spin term of k_K's numerator.
template <int Q>
__device__ __forceinline__ float row_coord(const FaceLattice& L, int si, int pi) {
  float gx = (float)Gauss<Q>::x(0);
#pragma unroll
  for (int t = 1; t < Q; ++t)
    if (pi == t) gx = (float)Gauss<Q>::x(t);
  const float lo_i = si ? L.PI : L.i0, w_i = si ? L.wI1 : L.wI0;
  return fmaf(0.5f * w_i, gx, lo_i + 0.5f * w_i);
}
__device__ __forceinline__ void row_terms(const Consts<float>& C, const FaceLattice& L, float AIa, float& pRow,
                                          float& qRow, float& tRow) {
  const float XIa = AIa - L.cI;
  const float XI2 = XIa * XIa;
  pRow = L.pK + XI2;
  qRow = fmaf(L.qI, XI2, L.qK);
  tRow = L.tI * XIa;
}
// Column jb = sj * Q + pj: grid coordinate along J and the column terms.
template <int Q>
__device__ __forceinline__ float col_coord(const FaceLattice& L, int jb) {
  const int sub = jb >= Q ? 1 : 0, pj = jb - sub * Q;
  float gx = (float)Gauss<Q>::x(0);
#pragma unroll
  for (int t = 1; t < Q; ++t)
    if (pj == t) gx = (float)Gauss<Q>::x(t);
  const float lo_j = sub ? L.PJ : L.j0, hi_j = sub ? L.j0 + 1.f : L.PJ;
  return fmaf(0.5f * (hi_j - lo_j), gx, 0.5f * (lo_j + hi_j));
}
__device__ __forceinline__ void col_terms(const Consts<float>& C, const FaceLattice& L, float AJ, float& pJ,
                                          float& qJ, float& tJ) {
  const float XJ = AJ - L.cJ;
  pJ = XJ * XJ;
  qJ = L.qJ * pJ;
  tJ = L.tJ * XJ;
}

// Eq. 18 integrand at one node from its r^2 (scalar form, for the deferred nodes).
__device__ __forceinline__ float node_value(const Consts<float>& C, const FaceLattice& L, float r2, float q,
                                            float t) {
  if (!(r2 > 0.f)) return 1.f;  // the flat limit r = 0
  const float r = r2 * rsqrtf(r2);
  const float sig = fmaf(r2, r2, q);
  float fperp;
  if (L.K == 2) {
    fperp = __fdividef(C.two_m * r * (r2 - L.XK * L.XK), sig);
  } else {
    const float num = fmaf(r, L.XK, t);
    const float rho2 = r2 + C.a2;
    const float rho4 = rho2 * rho2;
    fperp = __fdividef(C.two_m * r * r2 * fmaf(-num, num, rho4), rho4 * sig);
  }
  const float v = 1.f + fperp;
  return v * rsqrtf(v);
}

// Means of t^i (i = 0..4) over [0, x] (lane x: x^i / (i+1)) and over [x, 1] (lane y:
// (1 + x + ... + x^i) / (i+1)): the integral of a monomial over a sub-interval is its width times
// this mean, so the areas below keep the relative precision of the widths x and 1 - x.
__device__ __forceinline__ void interval_means(float x, float2 M[5]) {
  float p = x, cum = 1.f + x;
  M[0] = f2(1.f);
  M[1] = mul2(make_float2(p, cum), f2(0.5f));
#pragma unroll
  for (int i = 2; i < 5; ++i) {
    p *= x;
    cum += p;
    M[i] = mul2(make_float2(p, cum), f2(1.f / (float)(i + 1)));
  }
}

// The four sub-rectangle AREAs of Eq. 18 in the face plane at fraction w along K of a cell, split
// at fractions (u, v) along (I, J), from the cell's polynomial fit t (the 5 float4 of one face
// orientation, layout at kAreaTableStride in common.cuh: term n enumerates, for j = 0..4, i = 0..4-j,
// the coefficients of w^0..w^(4-i-j) of u^i v^j).  With c_ij the fit's u^i v^j coefficient at w, the
// area over U x V is |U| |V| sum_ij c_ij mean_U(u^i) mean_V(v^j).
// A00 = [u,1] x [v,1], A10 = [0,u] x [v,1], A01 = [u,1] x [0,v], A11 = [0,u] x [0,v].
__device__ __forceinline__ void table_areas(const float4* __restrict__ t, float u, float v, float w, float& A00,
                                            float& A10, float& A01, float& A11) {
  float c[kFitTerms];
  // streaming loads (evicted from L1 and L2 first): a cell's fits serve its own particles only
  const float4 e = __ldcs(t);
  c[0] = e.x;
  c[1] = e.y;
  c[5] = e.z;
  c[15] = e.w;
  float hv[32];  // the FP16 terms in term order
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 w4 = __ldcs(reinterpret_cast<const uint4*>(t + 1 + q));
    const unsigned wd[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&wd[r]));
      hv[8 * q + 2 * r] = f.x;
      hv[8 * q + 2 * r + 1] = f.y;
    }
  }
  {
    int h = 0;
#pragma unroll
    for (int n = 0; n < kFitTerms; ++n)
      if (!fit_term_fp32(n)) c[n] = hv[h++];
  }
  float2 Mu[5], Mv[5];
  interval_means(u, Mu);
  interval_means(v, Mv);
  // R_j = sum_i c_ij(w) mean(u^i) over [0,u] (lane x) and [u,1] (lane y); c_ij(w) by Horner in w
  float2 R[5];
  int n = 0;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
#pragma unroll
    for (int i = 0; i + j < 5; ++i) {
      const int kmax = 4 - i - j;
      float cij = c[n + kmax];
#pragma unroll
      for (int k = kmax - 1; k >= 0; --k) cij = fmaf(cij, w, c[n + k]);
      n += kmax + 1;
      R[j] = i == 0 ? f2(cij) : fma2(f2(cij), Mu[i], R[j]);
    }
  }
  // sums over j against mean(v^j) over [0,v] (S0) and [v,1] (S1)
  float2 S0 = R[0], S1 = R[0];
#pragma unroll
  for (int j = 1; j < 5; ++j) {
    S0 = fma2(R[j], f2(Mv[j].x), S0);
    S1 = fma2(R[j], f2(Mv[j].y), S1);
  }
  const float wu = 1.f - u, wv = 1.f - v;
  A11 = S0.x * (u * v);
  A01 = S0.y * (wu * v);
  A10 = S1.x * (u * wv);
  A00 = S1.y * (wu * wv);
}

// FP32 deposit (the zig-zag split, fluxes and Eq. 18 weights of deposit() below) evaluated on a
// per-face node lattice: the Q x Q Gauss nodes of the four sub-rectangles of a face make a
// 2Q x 2Q lattice in (x^I, x^J), so node coordinates, their squares and the spin terms are
// formed once per face (column terms) or row (row terms), roots are v * rsqrt(v) and each node
// needs one reciprocal.  Adjacent nodes of a row go through the formula as a packed pair.
//   Integrand: 1 + f (1 - k_K^2) with f = 2 m r^3 / Sigma, Sigma = r^4 + a^2 z^2, and
//   1 - k_z^2 = (r^2 - z^2) / r^2;  1 - k_x^2 = (rho^4 - (r x - a y)^2) / rho^4,
//   1 - k_y^2 = (rho^4 - (r y + a x)^2) / rho^4,  rho^2 = r^2 + a^2.
// With (I, J) = (K+1, K+2) mod 3: K = 0 -> (x, y, z) = (x^K, x^I, x^J); K = 1 -> (x^J, x^K, x^I);
// K = 2 -> (x^I, x^J, x^K).
// Every node first takes the far-field form: for a particle outside the near radius every node
// has R > |a|, so the quartic takes its p = R^2 - a^2 > 0 branch and every root argument is
// positive.  With mixed (a warp-uniform flag) a node with p <= 0 or an FP32 r below r_fp64 is
// left out of the sums and marked; after the lattice each marked node is evaluated again -- the
// cancellation-free form of the root, then the FP64 policy (node_newton64 on FP64 p and q) where
// it applies; r = 0 gives the flat limit -- and added.  The main loop has no call in it.
template <int Q, bool TAB = false>
__device__ __forceinline__ void deposit_lattice(const Grid& g, const Fields<float>& F, const Consts<float>& C,
                                                const float x0[3], const float dx[3], float qg, float inv_dt,
                                                unsigned& flags, unsigned& n64, bool mixed, const JTile& jt,
                                                const float4* __restrict__ atab = nullptr) {
  static_assert(4 * Q * Q <= 64, "node mask");
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
    // fr: the segment midpoint's position within the segment's cell, from x0 - c (exact: the two are
    // within two cells of each other) plus the small offset, so that the sub-rectangle widths keep
    // FP32's relative precision instead of the absolute rounding of a grid coordinate (~4e-6 cells at
    // coordinates near 100); the midpoint itself is c + fr
    float dseg[3], fr[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      dseg[ax] = seg ? s2[ax] : s1[ax];
      fr[ax] = seg ? (x0[ax] - (float)c2[ax]) + (s1[ax] + 0.5f * s2[ax]) : (x0[ax] - (float)c1[ax]) + 0.5f * s1[ax];
    }
    const long long base = ((long long)cz * g.ny + cy) * g.nx + cx;
#pragma unroll 1
    for (int K = 0; K < 3; ++K) {
      const float dK = sel3(K, dseg[0], dseg[1], dseg[2]);
      if (dK == 0.f) continue;
      const float flux = qg * dK * inv_dt;
      const float frI = sel3(K, fr[1], fr[2], fr[0]), frJ = sel3(K, fr[2], fr[0], fr[1]);
      float A00, A10, A01, A11;  // sub-rectangle areas; a node's weight is the area opposite it
      if constexpr (TAB) {
        table_areas(atab + base * kAreaTableStride + 5 * K, frI, frJ, sel3(K, fr[0], fr[1], fr[2]), A00, A10,
                    A01, A11);
      } else {
        FaceLattice L;
        L.K = K;
        L.i0 = (float)sel3(K, cy, cz, cx);
        L.j0 = (float)sel3(K, cz, cx, cy);
        L.PK = (float)sel3(K, cx, cy, cz) + sel3(K, fr[0], fr[1], fr[2]);
        L.XK = L.PK - sel3(K, cen[0], cen[1], cen[2]);
        L.PI = L.i0 + frI;
        L.PJ = L.j0 + frJ;
        L.cI = sel3(K, cen[1], cen[2], cen[0]);
        L.cJ = sel3(K, cen[2], cen[0], cen[1]);
        // sub-interval 0 = [i0, PI], 1 = [PI, i0 + 1] (likewise in J)
        L.wI0 = frI;
        L.wI1 = 1.f - frI;
        const float wJ[2] = {frJ, 1.f - frJ};
        // Per node the quartic needs p = R^2 - a^2 and q = a^2 z^2, k_K's numerator the spin term
        // -a x^I (K = 0) or +a x^J (K = 1); z is x^K, x^I or x^J (K = 2, 1, 0).  Each of these is a
        // sum of a face constant, a row term and a column term.
        L.pK = L.XK * L.XK - C.a2;
        L.qK = K == 2 ? C.a2 * L.XK * L.XK : 0.f;
        L.qI = K == 1 ? C.a2 : 0.f;
        L.tI = K == 0 ? -C.a : 0.f;
        L.qJ = K == 0 ? C.a2 : 0.f;
        L.tJ = K == 1 ? C.a : 0.f;
        float2 pJ2[Q], qJ2[Q], tJ2[Q];
  #pragma unroll
        for (int k = 0; k < Q; ++k) {
          const float2 XJ = add2(make_float2(col_coord<Q>(L, 2 * k), col_coord<Q>(L, 2 * k + 1)), f2(-L.cJ));
          const float2 sq = mul2(XJ, XJ);
          pJ2[k] = mul2(f2(0.5f), sq);
          qJ2[k] = mul2(f2(L.qJ), sq);
          tJ2[k] = mul2(f2(L.tJ), XJ);
        }
        const float nzz = -(L.XK * L.XK);
        // acc[si][k]: lane-wise sums over the rows of sub-interval si, node pair k of a row
        float2 acc[2][Q];
  #pragma unroll
        for (int si = 0; si < 2; ++si)
  #pragma unroll
          for (int k = 0; k < Q; ++k) acc[si][k] = f2(0.f);
        unsigned long long slow = 0ull;  // marked nodes, bit (si * Q + pi) * 2Q + jb
  #pragma unroll 1
        for (int pi = 0; pi < Q; ++pi) {
          float gw = (float)Gauss<Q>::w(0);
  #pragma unroll
          for (int t = 1; t < Q; ++t)
            if (pi == t) gw = (float)Gauss<Q>::w(t);
  #pragma unroll
          for (int si = 0; si < 2; ++si) {
            float pRow, qRow, tRow;
            row_terms(C, L, row_coord<Q>(L, si, pi), pRow, qRow, tRow);
            const float2 pR = f2(0.5f * pRow), qR = f2(qRow), tR = f2(tRow);
  #pragma unroll
            for (int k = 0; k < Q; ++k) {
              // with h = p / 2 (the halves of the row and column terms, exact):
              // r^2 = h + sqrt(h^2 + q), the root's p > 0 form
              const float2 p = add2(pR, pJ2[k]);
              const float2 q = add2(qR, qJ2[k]);
              const float2 D2 = fma2(p, p, q);
              const float2 rD2 = rsqrt2(D2);  // 2 / D
              const float2 r2 = fma2(D2, rD2, p);
              const float2 ir = rsqrt2(r2);
              // at the root r^4 + a^2 z^2 = r^2 D, so f = 2 m r^3 / Sigma = 2 m r / D = m r rsqrt(D2)
              float2 v;
              if (K == 2) {
                // f (1 - z^2 / r^2) = m rsqrt(D2) (r^2 - z^2) / r
                v = fma2(mul2(mul2(f2(C.m), rD2), add2(r2, f2(nzz))), ir, f2(1.f));
              } else {
                // f (1 - k_K^2) with k_K = num / rho^2
                const float2 r = mul2(r2, ir);
                const float2 num = fma2(r, f2(L.XK), add2(tR, tJ2[k]));
                const float2 kK = mul2(num, rcp2(add2(r2, f2(C.a2))));
                const float2 omk2 = fma2(kK, make_float2(-kK.x, -kK.y), f2(1.f));
                v = fma2(mul2(mul2(f2(C.m), r), rD2), omk2, f2(1.f));
              }
              float2 rv = rsqrt2(v);
              if (mixed) {
                const int bit = (si * Q + pi) * 2 * Q + 2 * k;
                if (!(p.x > 0.f) || !(r2.x >= C.r2_fp64)) {
                  v.x = rv.x = 0.f;
                  slow |= 1ull << bit;
                }
                if (!(p.y > 0.f) || !(r2.y >= C.r2_fp64)) {
                  v.y = rv.y = 0.f;
                  slow |= 1ull << (bit + 1);
                }
              }
              if (Q == 2) {
                acc[si][k] = fma2(v, rv, acc[si][k]);  // unit Gauss weights
              } else {
                const float2 w = make_float2(gw * (float)Gauss<Q>::w((2 * k) % Q),
                                             gw * (float)Gauss<Q>::w((2 * k + 1) % Q));
                acc[si][k] = fma2(w, mul2(v, rv), acc[si][k]);
              }
            }
          }
        }
        // S[si][sj]: the weighted integrand sums of the four sub-rectangles
        float S[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  #pragma unroll
        for (int si = 0; si < 2; ++si)
  #pragma unroll
          for (int k = 0; k < Q; ++k) {
            S[si][(2 * k) >= Q ? 1 : 0] += acc[si][k].x;
            S[si][(2 * k + 1) >= Q ? 1 : 0] += acc[si][k].y;
          }
        // The marked nodes of FP32-mixed warps.  p and q in FP64 are sums of FP64 face, row and
        // column terms, like their FP32 counterparts: face, row and column terms are formed once.
        if (slow) {
          const double cK = sel3(K, C.dxc, C.dyc, C.dzc), cI = sel3(K, C.dyc, C.dzc, C.dxc);
          const double cJ = sel3(K, C.dzc, C.dxc, C.dyc);
          const double XK64 = widen(L.PK) - cK;
          const double pK64 = fma(XK64, XK64, -C.da2);
          const double qK64 = K == 2 ? C.da2 * XK64 * XK64 : 0.0;
          double sqJ[2 * Q];  // squared FP64 offsets of the columns
  #pragma unroll
          for (int jb = 0; jb < 2 * Q; ++jb) {
            const double XJ64 = widen(col_coord<Q>(L, jb)) - cJ;
            sqJ[jb] = XJ64 * XJ64;
          }
          int row = -1;
          double pRow64 = 0.0, qRow64 = 0.0;
          do {
            const int b = __ffsll((long long)slow) - 1;
            slow &= slow - 1ull;
            const int ia = b / (2 * Q), jb = b - ia * 2 * Q;
            const int si = ia / Q, pi = ia - si * Q;
            const float AIa = row_coord<Q>(L, si, pi), AJ = col_coord<Q>(L, jb);
            float pRow, qRow, tRow, pJ, qJ, tJ;
            row_terms(C, L, AIa, pRow, qRow, tRow);
            col_terms(C, L, AJ, pJ, qJ, tJ);
            const float p = pRow + pJ, q = qRow + qJ;
            // FP32 root by the cancellation-free form; FP64 where the policy asks for it (a node
            // with p > 0 was marked only for that)
            const float D = sqrtf(fmaf(p, p, 4.f * q));
            float r2 = p >= 0.f ? 0.5f * (p + D) : __fdividef(2.f * q, D - p);
            if (p > 0.f || !(r2 >= C.r2_fp64)) {
              if (ia != row) {
                row = ia;
                const double XI64 = widen(AIa) - cI;
                pRow64 = fma(XI64, XI64, pK64);
                qRow64 = K == 1 ? C.da2 * XI64 * XI64 : qK64;
              }
              double sq = sqJ[0];
  #pragma unroll
              for (int t = 1; t < 2 * Q; ++t)
                if (jb == t) sq = sqJ[t];
              const double p64 = pRow64 + sq;
              const double q64 = K == 0 ? C.da2 * sq : qRow64;
              r2 = node_newton64(p64, q64, r2, D);
              ++n64;
            }
            float w = (float)Gauss<Q>::w(0), wj = (float)Gauss<Q>::w(0);
  #pragma unroll
            for (int t = 1; t < Q; ++t) {
              if (pi == t) w = (float)Gauss<Q>::w(t);
              if (jb % Q == t) wj = (float)Gauss<Q>::w(t);
            }
            const float add = w * wj * node_value(C, L, r2, q, tRow + tJ);
            const int sj = jb >= Q ? 1 : 0;
            S[0][0] += (si == 0 && sj == 0) ? add : 0.f;
            S[0][1] += (si == 0 && sj == 1) ? add : 0.f;
            S[1][0] += (si == 1 && sj == 0) ? add : 0.f;
            S[1][1] += (si == 1 && sj == 1) ? add : 0.f;
          } while (slow);
        }
        const float wI[2] = {L.wI0, L.wI1};
        A00 = S[1][1] * 0.25f * wI[1] * wJ[1];
        A10 = S[0][1] * 0.25f * wI[0] * wJ[1];
        A01 = S[1][0] * 0.25f * wI[1] * wJ[0];
        A11 = S[0][0] * 0.25f * wI[0] * wJ[0];
      }
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

// A load that the compiler may neither hoist nor merge with an earlier one: push_particle reads
// x_n and u_n again at every RK4 stage (they stay in L1) instead of holding them in registers
// across the stage evaluations, which leaves registers for more resident warps.
__device__ __forceinline__ float reload(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double reload(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// The move of a particle-step, which is all the deposit needs: x_n, the increment, q gamma-bar and
// whether to deposit at all (finite state, charged species).
template <typename T>
struct Move {
  T x0[3], dx[3], qg;
  bool go;
};

// One particle-step of particle i without its deposit (push_particle below, up to the deposit).
template <typename T, int Q>
__device__ __forceinline__ Move<T> push_move(const Grid& g, const Fields<T>& F, const Particles<T>& P,
                                             const Consts<T>& C, long long i, DevStatus* st, unsigned& flags,
                                             unsigned& n64, uint32_t* key_out, bool mixed) {
  // RK4 in proper time: stages at offsets 0, h/2, h/2, h; h = dt / gamma_1 (Eq. 16).  x^4 does
  // not enter a~ (the metric is stationary), so the stages carry x^1..x^3 only.
  T xs[3], us[4], a[4], sx[4], su[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < 3) xs[q] = P.x[q][i];
    us[q] = P.u[q][i];
    sx[q] = T(0);
    su[q] = T(0);
  }
  T h = T(0);
  bool fb = false;
#pragma unroll 1
  for (int stage = 0; stage < 4; ++stage) {
    accel<T>(g, F, C, xs, us, a, flags, n64, mixed);
    if (stage == 0) h = C.dt / gamma_step<T>(us[3], a[3], C.inv_c, C.dt, &fb);
    const T wgt = (stage == 0 || stage == 3) ? T(1) : T(2);
    const T frac = (stage == 2) ? h : T(0.5) * h;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sx[q] += wgt * us[q];
      su[q] += wgt * a[q];
      if (q < 3) xs[q] = reload(P.x[q] + i) + frac * us[q];
      us[q] = reload(P.u[q] + i) + frac * a[q];
    }
  }
  T x0[3], x1[4], u1[4], dx[3];
  const T h6 = h / T(6);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T xq = reload(P.x[q] + i), d = h6 * sx[q];
    if (q < 3) {
      x0[q] = xq;
      dx[q] = d;
    }
    x1[q] = xq + d;
    u1[q] = reload(P.u[q] + i) + h6 * su[q];
  }
  x1[3] -= C.cdt;  // x^4 is stored relative to c t
  const T gbar = C.gamma_in_j ? (reload(P.u[3] + i) + u1[3]) / (T(2) * C.c) : T(1);
  bool finite = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) finite = finite && isfinite(x1[q]) && isfinite(u1[q]);
  if (!finite) flags |= ST_NONFINITE;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (!(fabs(x1[q] - x0[q]) < T(1))) flags |= ST_CFL;
  // streaming (evict-first) stores: the new state is read again only by the next step or the sort
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __stcs(P.x[q] + i, x1[q]);
    __stcs(P.u[q] + i, u1[q]);
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
    __stcs(key_out, kDead);
    atomicAdd(horizon ? &st->removed_horizon : &st->removed_outer, 1ull);
  } else {
    const int ci = (int)floor(x1[0]), cj = (int)floor(x1[1]), ck = (int)floor(x1[2]);
    __stcs(key_out, (uint32_t)(((long long)ck * g.ny + cj) * g.nx + ci));
  }
  if (fb) atomicAdd(&st->fallbacks, 1ull);
  Move<T> mv;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    mv.x0[q] = x0[q];
    mv.dx[q] = dx[q];
  }
  mv.qg = C.qmacro * gbar;  // J = rho gamma v
  mv.go = finite && C.qmacro != T(0);
  return mv;
}

// The deposit of a move (Sec. 4).  TAB (far-field warps, T = float): face areas from the per-cell
// fits atab.
template <typename T, int Q, bool TAB = false>
__device__ __forceinline__ void deposit_move(const Grid& g, const Fields<T>& F, const Consts<T>& C, const Move<T>& mv,
                                             unsigned& flags, unsigned& n64, bool mixed, const JTile& jt = JTile(),
                                             const float4* atab = nullptr) {
  if (!mv.go) return;
  if constexpr (sizeof(T) == sizeof(float))
    deposit_lattice<Q, TAB>(g, F, C, mv.x0, mv.dx, mv.qg, C.inv_dt, flags, n64, mixed, jt, atab);
  else
    deposit<T, Q>(g, F, C, mv.x0, mv.dx, mv.qg, C.inv_dt, flags);
}

// One particle-step of particle i: RK4 push, new state stored, removal flag and sort key
// (written to *key_out: P.key + i, or a side array where another kernel still reads P.key
// concurrently), then the deposit of the move (which needs only x_n and the increment).
// mixed (T = float): the FP32-mixed policy applies to this warp's particles (a warp-uniform
// flag; false only where every particle lies outside near_radius).  T = double ignores it.
// TAB (far-field warps, T = float): the deposit takes its face areas from the per-cell fits atab.
template <typename T, int Q, bool TAB = false>
__device__ __forceinline__ void push_particle(const Grid& g, const Fields<T>& F, const Particles<T>& P,
                                              const Consts<T>& C, long long i, DevStatus* st, unsigned& flags,
                                              unsigned& n64, uint32_t* key_out, bool mixed,
                                              const JTile& jt = JTile(), const float4* atab = nullptr) {
  const Move<T> mv = push_move<T, Q>(g, F, P, C, i, st, flags, n64, key_out, mixed);
  deposit_move<T, Q, TAB>(g, F, C, mv, flags, n64, mixed, jt, atab);
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
