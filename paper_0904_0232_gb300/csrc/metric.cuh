// Device metric module for the Cartesian Kerr-Schild form of the Kerr metric.
//
//   g_mn = eta_mn + f k_m k_n,   f = 2 m r^3 / (r^4 + a^2 z^2)                 (Eq. 4)
//   k = ((r x - a y)/(r^2 + a^2), (r y + a x)/(r^2 + a^2), z / r, 1)          (Eq. 5, dt -> dx^4)
//   r^4 - (R^2 - a^2) r^2 - a^2 z^2 = 0                                        (Eq. 6)
//
// k is null for eta (that is Eq. 6), so |k_spatial| = 1, det g = -1 and
// g^mn = eta^mn - f k^m k^n with k^m = (k_x, k_y, k_z, -1).  Everything below uses those
// closed forms; the gradients of r, f and k are written out by the chain rule.
#pragma once

#include <cuda_runtime.h>

namespace grpic {

// Division and square root used by the metric functions.  IeeeOps is the compiler's own
// operators (the default everywhere); a caller that needs less than full precision can pass a
// cheaper policy with the same three members.
struct IeeeOps {
  template <typename S>
  __device__ static __forceinline__ S rcp(S x) { return S(1) / x; }
  template <typename S>
  __device__ static __forceinline__ S div(S a, S b) { return a / b; }
  template <typename S>
  __device__ static __forceinline__ S root(S x) { return sqrt(x); }
};

// IEEE 754 binary32 -> binary64, exact, with integer operations only (sign, exponent rebiased
// by 1023 - 127 = 896, mantissa shifted by 29).  Zero and subnormal inputs give a signed zero
// (the FP32 push runs with subnormals flushed); infinities and NaNs keep their class.  On this
// GPU the hardware conversions run on the reduced-rate FP64 pipe.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned hi = u & 0x80000000u, lo = 0u;
  if (e != 0u) {
    const unsigned m = u & 0x7fffffu;
    hi |= ((e == 0xffu ? 0x7ffu : e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// IEEE 754 binary64 -> binary32 with round-to-nearest-even, with integer operations for every
// result in the normal binary32 range (the 29 dropped mantissa bits decide; a carry may step the
// exponent, to infinity at the top, as the rounding rule says) and for zeros; other inputs
// (subnormal or out-of-range results, infinities, NaNs) take the hardware conversion.
__device__ __forceinline__ float narrow(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e == 0u && (hi & 0xfffffu) == 0u && lo == 0u) return __uint_as_float(hi & 0x80000000u);  // +-0
  if (e < 897u || e > 1150u) return __double2float_rn(d);
  unsigned r = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ++r;
  return __uint_as_float(r);
}

// FP64 reciprocal, quotient and square root for evaluations whose results are rounded to FP32
// afterwards (the FP32-mixed policy near the hole), where IEEE rounding of the last FP64 bit
// buys nothing: an FP32 estimate (the approximate reciprocal / reciprocal square root, relative
// error a few 2^-23) refined by one FP64 Newton step -- y <- y + y (1 - x y) for 1/x, and
// s <- s + (x - s^2) y / 2 with s = x y, y ~ 1/sqrt x, for sqrt x (Heron).  A Newton step
// squares the relative error.  Arguments outside [1e-30, 1e30] in magnitude (and non-positive
// square-root arguments) take the IEEE operations.
struct SeededOps64 {
  __device__ static __forceinline__ double rcp(double x) {
    const float xf = narrow(x);
    if (!(fabsf(xf) >= 1e-30f && fabsf(xf) <= 1e30f)) return 1.0 / x;
    const double y = widen(__fdividef(1.f, xf));
    return fma(y, fma(-x, y, 1.0), y);
  }
  __device__ static __forceinline__ double div(double a, double b) { return a * rcp(b); }
  __device__ static __forceinline__ double root(double x) {
    const float xf = narrow(x);
    if (!(xf >= 1e-30f && xf <= 1e30f)) return sqrt(x);
    const double y = widen(rsqrtf(xf));
    const double s = x * y;
    return fma(0.5 * y, fma(-s, s, x), s);
  }
};

template <typename S>
struct Kerr {
  S r, f;        // r of Eq. 6, f of Eq. 4
  S k0, k1, k2;  // spatial k_m (k_3 = 1)
  S D;           // sqrt((R^2 - a^2)^2 + 4 a^2 z^2) = d(quartic)/d(r^2)
  S inv_r, inv_rho2, inv_sig, inv_D;  // 1/r, 1/(r^2 + a^2), 1/(r^4 + a^2 z^2), 1/D, shared with the derivatives
  bool flat;     // r = 0 (the disk z = 0, R <= a): metric taken flat, its limit there
};

// Non-negative root of Eq. 6 as r^2, written so that neither branch cancels; *D receives
// sqrt((R^2 - a^2)^2 + 4 a^2 z^2).
template <typename S, typename Ops = IeeeOps>
__device__ __forceinline__ S kerr_r2(S x, S y, S z, S a, S* D) {
  const S a2 = a * a;
  const S q = a2 * z * z;
  const S p = x * x + y * y + z * z - a2;
  *D = Ops::root(p * p + S(4) * q);
  return (p >= S(0)) ? S(0.5) * (p + *D) : Ops::div(S(2) * q, *D - p);
}

// f and k of Eqs. 4-5 at (x, y, z) given r^2 from Eq. 6.
template <typename S, typename Ops = IeeeOps>
__device__ __forceinline__ Kerr<S> kerr_from_r2(S x, S y, S z, S m, S a, S r2, S D) {
  Kerr<S> K;
  const S a2 = a * a;
  const S q = a2 * z * z;
  K.D = D;
  if (!(r2 > S(0))) {
    K.flat = true;
    K.r = S(0);
    K.f = S(0);
    K.k0 = S(0);
    K.k1 = S(0);
    K.k2 = S(1);
    return K;
  }
  K.flat = false;
  K.r = Ops::root(r2);
  K.inv_r = Ops::rcp(K.r);
  K.inv_rho2 = Ops::rcp(r2 + a2);
  K.inv_sig = Ops::rcp(r2 * r2 + q);
  K.inv_D = Ops::rcp(D);
  K.f = S(2) * m * K.r * r2 * K.inv_sig;
  K.k0 = (K.r * x - a * y) * K.inv_rho2;
  K.k1 = (K.r * y + a * x) * K.inv_rho2;
  K.k2 = z * K.inv_r;
  return K;
}

// Integrand of Eq. 18 for the plane normal to axis K: g_II g_JJ - g_IJ^2 = 1 + f (k_I^2 + k_J^2)
// and, k being null for eta (Eq. 6), k_I^2 + k_J^2 = 1 - k_K^2.  Given r^2 from Eq. 6.
template <typename S>
__device__ __forceinline__ S area_density(S x, S y, S z, S m, S a, S r2, int K) {
  if (!(r2 > S(0))) return S(1);
  const S r = sqrt(r2);
  const S a2 = a * a;
  const S sig = r2 * r2 + a2 * z * z;
  if (K == 2) {
    // f (1 - z^2/r^2) = 2 m r (r^2 - z^2) / Sigma
    return sqrt(S(1) + S(2) * m * r * (r2 - z * z) / sig);
  }
  // f (1 - k_K^2) with k_x = (r x - a y)/(r^2+a^2), k_y = (r y + a x)/(r^2+a^2)
  const S num = (K == 0) ? (r * x - a * y) : (r * y + a * x);
  const S rho2 = r2 + a2;
  const S kk = num * num / (rho2 * rho2);
  return sqrt(S(1) + S(2) * m * r * r2 * (S(1) - kk) / sig);
}

template <typename S, typename Ops = IeeeOps>
__device__ __forceinline__ Kerr<S> kerr_eval(S x, S y, S z, S m, S a) {
  S D;
  const S r2 = kerr_r2<S, Ops>(x, y, z, a, &D);
  return kerr_from_r2<S, Ops>(x, y, z, m, a, r2, D);
}

// Gamma^a_mn u^m u^n = g^ab (u^m d_m g_bn u^n - 1/2 d_b g_mn u^m u^n) for g = eta + f k k.
// With s = k.u, D_b = u^m d_m k_b, E_b = u^n d_b k_n and d_4 = 0:
//   w_b = (u.df) s k_b + f s D_b + f (u.D) k_b - 1/2 s^2 d_b f - f s E_b
//   Gamma u u = eta^ab w_b - f k^a (k^b w_b)
template <typename S, typename Ops = IeeeOps>
__device__ __forceinline__ void christoffel_uu(const Kerr<S>& K, S x, S y, S z, S a, const S u[4], S out[4]) {
  if (K.flat) {
    out[0] = out[1] = out[2] = out[3] = S(0);
    return;
  }
  const S r = K.r, f = K.f;
  const S k0 = K.k0, k1 = K.k1, k2 = K.k2;
  const S r2 = r * r, a2 = a * a;
  const S inv_rho2 = K.inv_rho2;
  const S inv_D = K.inv_D;
  const S inv_r = K.inv_r;
  // grad r from the implicit quartic: r_x = x r / D, r_y = y r / D, r_z = z (r^2 + a^2) / (r D)
  const S rx = x * r * inv_D;
  const S ry = y * r * inv_D;
  const S rz = z * (r2 + a2) * inv_D * inv_r;
  // grad f: df/dr = f (3/r - 4 r^3/Sigma), df/dz|_r = -2 a^2 z f / Sigma, Sigma = r^4 + a^2 z^2
  const S inv_sig = K.inv_sig;
  const S fr = f * (S(3) * inv_r - S(4) * r2 * r * inv_sig);
  const S fx = fr * rx;
  const S fy = fr * ry;
  const S fz = fr * rz - S(2) * a2 * z * f * inv_sig;
  // Jacobian J[i][j] = d_i k_j
  const S ri[3] = {rx, ry, rz};
  S Jk[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const S tr = S(2) * r * ri[i];
    Jk[i][0] = (x * ri[i] + (i == 0 ? r : S(0)) - (i == 1 ? a : S(0)) - tr * k0) * inv_rho2;
    Jk[i][1] = (y * ri[i] + (i == 1 ? r : S(0)) + (i == 0 ? a : S(0)) - tr * k1) * inv_rho2;
    Jk[i][2] = ((i == 2 ? S(1) : S(0)) - k2 * ri[i]) * inv_r;
  }
  const S s = k0 * u[0] + k1 * u[1] + k2 * u[2] + u[3];
  const S uf = u[0] * fx + u[1] * fy + u[2] * fz;
  S Dv[3], Ev[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    Dv[j] = u[0] * Jk[0][j] + u[1] * Jk[1][j] + u[2] * Jk[2][j];
    Ev[j] = u[0] * Jk[j][0] + u[1] * Jk[j][1] + u[2] * Jk[j][2];
  }
  const S uD = u[0] * Dv[0] + u[1] * Dv[1] + u[2] * Dv[2];
  const S fg[3] = {fx, fy, fz};
  const S kv[3] = {k0, k1, k2};
  const S c1 = uf * s + f * uD;  // coefficient of k_b in w_b (and w_4 itself)
  const S fs = f * s;
  const S hs2 = S(0.5) * s * s;
  S w[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) w[j] = c1 * kv[j] + fs * (Dv[j] - Ev[j]) - hs2 * fg[j];
  const S w3 = c1;
  const S kw = k0 * w[0] + k1 * w[1] + k2 * w[2] - w3;
  out[0] = w[0] - f * k0 * kw;
  out[1] = w[1] - f * k1 * kw;
  out[2] = w[2] - f * k2 * kw;
  out[3] = -w3 + f * kw;
}

// Field tensor at a point from the prognostic pair: covariant b = (F_yz, F_zx, F_xy) and
// contravariant d = (F^x4, F^y4, F^z4).  Lowering F with g = eta + f k k gives, for the
// spatial block, F_cov = M F^sp M + f (d k^T - k d^T) with M = I + f k k^T, so
//   alpha = b - f (d x k),  h = (F^yz, F^zx, F^xy) = [alpha + f k (k.alpha)] / (1 + f),
// and the covariant electric part e_i = F_i4 = f (k x h)_i + (f - 1) d_i - f k_i (k.d).
template <typename S>
__device__ __forceinline__ void contra_spatial(S f, S k0, S k1, S k2, const S b[3], const S d[3], S h[3]) {
  const S al0 = b[0] - f * (d[1] * k2 - d[2] * k1);
  const S al1 = b[1] - f * (d[2] * k0 - d[0] * k2);
  const S al2 = b[2] - f * (d[0] * k1 - d[1] * k0);
  const S ka = f * (k0 * al0 + k1 * al1 + k2 * al2);
  const S inv = S(1) / (S(1) + f);
  h[0] = (al0 + ka * k0) * inv;
  h[1] = (al1 + ka * k1) * inv;
  h[2] = (al2 + ka * k2) * inv;
}

template <typename S>
__device__ __forceinline__ void cov_electric(S f, S k0, S k1, S k2, const S h[3], const S d[3], S e[3]) {
  const S kd = k0 * d[0] + k1 * d[1] + k2 * d[2];
  const S fm1 = f - S(1);
  e[0] = f * (k1 * h[2] - k2 * h[1]) + fm1 * d[0] - f * k0 * kd;
  e[1] = f * (k2 * h[0] - k0 * h[2]) + fm1 * d[1] - f * k1 * kd;
  e[2] = f * (k0 * h[1] - k1 * h[0]) + fm1 * d[2] - f * k2 * kd;
}

// Lorentz part of Eq. 15, (q/m) F^a_b u^b = (q/m) F^ac u_c, with u_c = g_cb u^b:
//   u_i = u^i + f s k_i, u_4 = -u^4 + f s;  (q/m)[(u_cov x h)_i + d_i u_4],  -(q/m) d.u_cov
template <typename S>
__device__ __forceinline__ void lorentz(S qm, S f, S k0, S k1, S k2, const S h[3], const S d[3], const S u[4],
                                        S out[4]) {
  const S s = k0 * u[0] + k1 * u[1] + k2 * u[2] + u[3];
  const S fs = f * s;
  const S c0 = u[0] + fs * k0, c1 = u[1] + fs * k1, c2 = u[2] + fs * k2;
  const S c3 = fs - u[3];
  out[0] = qm * (c1 * h[2] - c2 * h[1] + d[0] * c3);
  out[1] = qm * (c2 * h[0] - c0 * h[2] + d[1] * c3);
  out[2] = qm * (c0 * h[1] - c1 * h[0] + d[2] * c3);
  out[3] = -qm * (d[0] * c0 + d[1] * c1 + d[2] * c2);
}

// Covariant spatial block of a contravariant tensor given as (h, d): with v_i = F^{i b} k_b,
// (g F g)_ij = F^ij + f (v_i k_j - k_i v_j).  Returns (F_yz, F_zx, F_xy).
template <typename S>
__device__ __forceinline__ void lower_spatial(S f, S k0, S k1, S k2, const S h[3], const S d[3], S b[3]) {
  // F^{ij} k_j = (k x h) components with sign: F^{il} k_l = eps_ilm k_l h_m = (k x h)_i
  const S v0 = (k1 * h[2] - k2 * h[1]) + d[0];
  const S v1 = (k2 * h[0] - k0 * h[2]) + d[1];
  const S v2 = (k0 * h[1] - k1 * h[0]) + d[2];
  b[0] = h[0] + f * (v1 * k2 - k1 * v2);
  b[1] = h[1] + f * (v2 * k0 - k2 * v0);
  b[2] = h[2] + f * (v0 * k1 - k0 * v1);
}

// Eq. 16: gamma = [u^4/c + sqrt((u^4/c)^2 + 4 a^4 dt / (2c))] / 2; a negative argument or a
// non-positive result falls back to u^4/c (the caller counts it).
template <typename S>
__device__ __forceinline__ S gamma_step(S u4, S a4, S inv_c, S dt, bool* fallback) {
  const S w = u4 * inv_c;
  const S arg = w * w + S(2) * a4 * dt * inv_c;
  S g = S(-1);
  if (arg >= S(0)) g = S(0.5) * (w + sqrt(arg));
  if (!(g > S(0))) {
    *fallback = true;
    return w;
  }
  *fallback = false;
  return g;
}

}  // namespace grpic
