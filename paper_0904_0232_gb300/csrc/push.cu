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
#include <algorithm>
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

struct Consts {
  double m, a, xc, yc, zc;
  float r_fp64;  // FP32-mixed: evaluate in FP64 where the FP32 r is below this
};

template <typename T>
__device__ __forceinline__ T sel3(int i, T a, T b, T c) {
  return i == 0 ? a : (i == 1 ? b : c);
}

// FP64 metric and Christoffel contraction at a grid position (the FP32-mixed policy near the
// hole); kept out of line: it runs for few particles and would otherwise bloat every call site.
template <typename T>
__device__ __noinline__ void metric_christoffel_fp64(const Consts& C, T x, T y, T z, T u0, T u1, T u2, T u3,
                                                     T* out) {
  const double Xd = (double)x - C.xc, Yd = (double)y - C.yc, Zd = (double)z - C.zc;
  const Kerr<double> K = kerr_eval<double>(Xd, Yd, Zd, C.m, C.a);
  const double ud[4] = {(double)u0, (double)u1, (double)u2, (double)u3};
  double gd[4];
  christoffel_uu<double>(K, Xd, Yd, Zd, C.a, ud, gd);
  out[0] = (T)K.f;
  out[1] = (T)K.k0;
  out[2] = (T)K.k1;
  out[3] = (T)K.k2;
  out[4] = (T)gd[0];
  out[5] = (T)gd[1];
  out[6] = (T)gd[2];
  out[7] = (T)gd[3];
}

// FP64 root of the quartic (Eq. 6) as r^2 and D, for quadrature nodes near the hole.
template <typename T>
__device__ __noinline__ void quartic_fp64(const Consts& C, T x, T y, T z, T* r2, T* D) {
  double Dd;
  const double r2d = kerr_r2<double>((double)x - C.xc, (double)y - C.yc, (double)z - C.zc, C.a, &Dd);
  *r2 = (T)r2d;
  *D = (T)Dd;
}

// a~ at (x, u): gather, convert, Lorentz - Christoffel.
template <typename T, bool MIXED>
__device__ __forceinline__ void accel(const Grid& g, const Fields<T>& F, const Consts& C, T qm, const T x[3],
                                      const T u[4], T out[4], unsigned& flags, unsigned& n64) {
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
    const long long base = ((long long)k0 * g.ny + j0) * g.nx + i0;
    T s = T(0);
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
          const T W = (di ? w0 : T(1) - w0) * (dj ? w1 : T(1) - w1) * (dk ? w2 : T(1) - w2);
          s += W * __ldg(arr + base + dk * sz + dj * sy + di);
        }
    val[comp] = s;
  }
  const T d[3] = {val[0], val[1], val[2]};
  const T b[3] = {val[3], val[4], val[5]};

  // --- metric and Christoffel contraction at the particle
  T f, k0, k1, k2, gam[4];
  const T X = x[0] - (T)C.xc, Y = x[1] - (T)C.yc, Z = x[2] - (T)C.zc;
  const Kerr<T> Kt = kerr_eval<T>(X, Y, Z, (T)C.m, (T)C.a);
  if (MIXED && (float)Kt.r < C.r_fp64) {
    T o[8];
    metric_christoffel_fp64<T>(C, x[0], x[1], x[2], u[0], u[1], u[2], u[3], o);
    f = o[0];
    k0 = o[1];
    k1 = o[2];
    k2 = o[3];
    gam[0] = o[4];
    gam[1] = o[5];
    gam[2] = o[6];
    gam[3] = o[7];
    ++n64;
  } else {
    christoffel_uu<T>(Kt, X, Y, Z, (T)C.a, u, gam);
    f = Kt.f;
    k0 = Kt.k0;
    k1 = Kt.k1;
    k2 = Kt.k2;
  }
  T h[3], lor[4];
  contra_spatial(f, k0, k1, k2, b, d, h);
  lorentz(qm, f, k0, k1, k2, h, d, u, lor);
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = lor[q] - gam[q];
}

// Integrand of Eq. 18, sqrt(g_II g_JJ - g_IJ^2) = sqrt(1 + f (k_I^2 + k_J^2)), at a grid
// position.  FP32-mixed: near the hole the quartic root is taken in FP64.
template <typename T, bool MIXED>
__device__ __forceinline__ T area_integrand(const Consts& C, T px, T py, T pz, int K, unsigned& n64) {
  const T X = px - (T)C.xc, Y = py - (T)C.yc, Z = pz - (T)C.zc;
  T D;
  T r2 = kerr_r2<T>(X, Y, Z, (T)C.a, &D);
  if (MIXED && (float)r2 < C.r_fp64 * C.r_fp64) {
    quartic_fp64<T>(C, px, py, pz, &r2, &D);
    ++n64;
  }
  return area_density<T>(X, Y, Z, (T)C.m, (T)C.a, r2, K);
}

// AREA of Eq. 18 over [Is, If] x [Js, Jf] in the plane x^K = xK.
template <typename T, int Q, bool MIXED>
__device__ __forceinline__ T area(const Consts& C, int K, T xK, T Is, T If, T Js, T Jf, unsigned& n64) {
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
      s += (T)Gauss<Q>::w(p) * (T)Gauss<Q>::w(q) * area_integrand<T, MIXED>(C, px, py, pz, K, n64);
    }
  return s * T(0.25) * (If - Is) * (Jf - Js);
}

// Umeda zig-zag deposit of the move x0 -> x0 + dx.  The segment displacements are carried
// as offsets from x0 (s1 = relay - x0, s2 = dx - s1), so the flux keeps the accuracy of the RK4
// increment instead of inheriting the rounding of the stored positions.  With |dx| < 1 the
// relay point min(min(a,b)+1, max(max(a,b), mid)) is the midpoint when the cell does not
// change along an axis and the shared face otherwise.
template <typename T, int Q, bool MIXED>
__device__ __forceinline__ void deposit(const Grid& g, const Fields<T>& F, const Consts& C, const T x0[3],
                                        const T dx[3], T qg, T inv_dt, unsigned& flags, unsigned& n64) {
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
      const T A00 = area<T, Q, MIXED>(C, K, PK, PI, i0 + T(1), PJ, j0 + T(1), n64);
      const T A10 = area<T, Q, MIXED>(C, K, PK, i0, PI, PJ, j0 + T(1), n64);
      const T A01 = area<T, Q, MIXED>(C, K, PK, PI, i0 + T(1), j0, PJ, n64);
      const T A11 = area<T, Q, MIXED>(C, K, PK, i0, PI, j0, PJ, n64);
      const T FA = A00 + A10 + A01 + A11;
      const T W00 = A00 / FA, W10 = A10 / FA, W01 = A01 / FA, W11 = A11 / FA;
      const long long stI = sel3(K, sy, sz, 1ll), stJ = sel3(K, sz, 1ll, sy);
      double* JK = sel3(K, F.J[0], F.J[1], F.J[2]);
      atomicAdd(JK + base, (double)(flux * W00));
      atomicAdd(JK + base + stI, (double)(flux * W10));
      atomicAdd(JK + base + stJ, (double)(flux * W01));
      atomicAdd(JK + base + stI + stJ, (double)(flux * W11));
    }
  }
}

// One particle-step of particle i: RK4 push, deposit, removal flag and sort key.
template <typename T, int Q, bool MIXED>
__device__ __forceinline__ void push_particle(const Grid& g, const Fields<T>& F, const Particles<T>& P,
                                              const Species& sp, long long i, DevStatus* st, unsigned& flags,
                                              unsigned& n64) {
  {
    Consts C;
    C.m = g.m;
    C.a = g.a;
    C.xc = g.xc;
    C.yc = g.yc;
    C.zc = g.zc;
    C.r_fp64 = (float)g.r_fp64;
    const T qm = (T)sp.qm;
    const T dt = (T)g.dt;
    T x0[4], u0[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      x0[q] = P.x[q][i];
      u0[q] = P.u[q][i];
    }
    // RK4 in proper time (A1): stages at offsets 0, h/2, h/2, h; h = dt / gamma_1 (Eq. 16)
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
      accel<T, MIXED>(g, F, C, qm, xs, us, a, flags, n64);
      if (stage == 0) h = dt / gamma_step<T>(u0[3], a[3], T(1) / (T)g.c, dt, &fb);
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
    x1[3] -= (T)(g.c * g.dt);  // x^4 is stored relative to c t
    bool finite = true;
#pragma unroll
    for (int q = 0; q < 4; ++q) finite = finite && isfinite(x1[q]) && isfinite(u1[q]);
    if (!finite) flags |= ST_NONFINITE;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (!(fabs(x1[q] - x0[q]) < T(1))) flags |= ST_CFL;
    // deposit, J = rho gamma v
    if (finite && sp.qmacro != 0.0) {
      const T gbar = (g.flags & 1u) ? T(1) : (u0[3] + u1[3]) / (T(2) * (T)g.c);
      const T qg = (T)sp.qmacro * gbar;
      deposit<T, Q, MIXED>(g, F, C, x0, dx, qg, T(1) / dt, flags, n64);
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
    if (finite && g.m > 0.0) {
      // cheap FP32 screen, FP64 decision near r_+
      const T X = x1[0] - (T)g.xc, Y = x1[1] - (T)g.yc, Z = x1[2] - (T)g.zc;
      T D;
      const T r2 = kerr_r2<T>(X, Y, Z, (T)g.a, &D);
      if ((double)r2 < 1.2 * g.r_plus * g.r_plus + 1.0) {
        double Dd;
        const double r2d =
            kerr_r2<double>((double)x1[0] - g.xc, (double)x1[1] - g.yc, (double)x1[2] - g.zc, g.a, &Dd);
        horizon = !(r2d > 0.0) || sqrt(r2d) <= g.r_plus;
      }
    }
    if (horizon || outer) {
      P.key[i] = kDead;
      atomicAdd(horizon ? &st->removed_horizon : &st->removed_outer, 1ull);
    } else {
      const int ci = (int)floor(x1[0]), cj = (int)floor(x1[1]), ck = (int)floor(x1[2]);
      P.key[i] = (uint32_t)(((long long)ck * g.ny + cj) * g.nx + ci);
    }
    if (fb) atomicAdd(&st->fallbacks, 1ull);
  }
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

template <typename T, int Q, bool MIXED>
__global__ void __launch_bounds__(128, 4) k_push_deposit(const Grid g, const Fields<T> F, const Particles<T> P,
                                                           const Species sp, DevStatus* st) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned flags = 0, n64 = 0;
  bool active = i < P.n && i < (long long)(*P.n_dev);
  if (active) active = P.key[i] != kDead;
  if (active) push_particle<T, Q, MIXED>(g, F, P, sp, i, st, flags, n64);
  warp_status(st, flags, n64, active);
}

// Batched: grid-stride over (instance * 4 + species, block) work items; each block belongs to
// one instance and species, so the warp-level status stays per instance.  The block's instance
// descriptor is staged in shared memory and reloaded only when the instance changes (a CTA's
// consecutive grid-stride blocks mostly stay inside one instance).
template <typename T, int Q, bool MIXED>
__global__ void __launch_bounds__(128, 4) k_push_deposit_batch(const InstDesc<T>* __restrict__ desc,
                                                                 const BlockEntry* __restrict__ blk, int nblk) {
  __shared__ Grid sg;
  __shared__ Fields<T> sF;
  __shared__ Particles<T> sP;
  __shared__ Species ssp;
  __shared__ DevStatus* sst;
  int loaded = -1;
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    const BlockEntry e = blk[bi];
    if (e.inst != loaded) {
      __syncthreads();
      if (threadIdx.x == 0) {
        const InstDesc<T>& D = desc[e.inst >> 2];
        const SpeciesDesc<T>& S = D.sp[e.inst & 3];
        sg = D.g;
        sF = D.F;
        sP = S.buf[*S.cur];
        ssp = Species{S.qm, S.qmacro};
        sst = D.st;
      }
      __syncthreads();
      loaded = e.inst;
    }
    const long long i = (long long)e.block * blockDim.x + threadIdx.x;
    unsigned flags = 0, n64 = 0;
    bool active = i < sP.n && i < (long long)(*sP.n_dev);
    if (active) active = sP.key[i] != kDead;
    if (active) push_particle<T, Q, MIXED>(sg, sF, sP, ssp, i, sst, flags, n64);
    warp_status(sst, flags, n64, active);
  }
}

// ---- load / unload ---------------------------------------------------------------------
template <typename T>
__global__ void k_load(const Grid g, const Particles<T> P, long long n, const double* __restrict__ x4,
                       const double* __restrict__ u4, const uint32_t* __restrict__ ids, int umode, double ct_now,
                       DevStatus* st) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x[3] = {x4[i], x4[n + i], x4[2 * n + i]};
  unsigned bad = 0;
  const int nn[3] = {g.nx, g.ny, g.nz};
  for (int q = 0; q < 3; ++q)
    if (!(x[q] >= 1.0 && x[q] <= nn[q] - 2)) bad |= ST_LOAD_INVALID;
  double u[4] = {u4[i], u4[n + i], u4[2 * n + i], umode == 0 ? u4[3 * n + i] : 0.0};
  // the removal rule (r <= r_+) applies from the start: such particles are dropped at load
  bool inside = false;
  if (!bad && g.m > 0.0) {
    const Kerr<double> K = kerr_eval<double>(x[0] - g.xc, x[1] - g.yc, x[2] - g.zc, g.m, g.a);
    inside = K.flat || K.r <= g.r_plus;
    if (inside) atomicAdd(&st->removed_horizon, 1ull);
  }
  if (!bad && !inside && umode != 0) {
    const Kerr<double> K = kerr_eval<double>(x[0] - g.xc, x[1] - g.yc, x[2] - g.zc, g.m, g.a);
    const double f = K.f, kk[4] = {K.k0, K.k1, K.k2, 1.0};
    const double c2 = g.c * g.c;
    if (umode == 1) {
      // covariant u_i given: g^mn u_m u_n = -c^2 with g^mn = eta^mn - f k^m k^n, k^m = (k_i, -1)
      // (-1 - f) u_4^2 + 2 (f k.u) u_4 + (|u|^2 - f (k.u)^2 + c^2) = 0, u^4 = g^{4n} u_n > 0
      const double ku = kk[0] * u[0] + kk[1] * u[1] + kk[2] * u[2];
      const double A = -1.0 - f, B = 2.0 * f * ku;
      const double Cc = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] - f * ku * ku + c2;
      const double disc = B * B - 4.0 * A * Cc;
      if (disc < 0.0) {
        bad |= ST_LOAD_INVALID;
      } else {
        // u^4 = g^{4n} u_n = -u_4 + f (k.u - u_4)  (k^4 = -1); pick the root with u^4 > 0
        const double sq = sqrt(disc);
        const double r1 = (-B + sq) / (2.0 * A), r2 = (-B - sq) / (2.0 * A);
        const double up1 = -r1 + f * (ku - r1), up2 = -r2 + f * (ku - r2);
        const double ul4 = (up1 > 0.0) ? r1 : r2;
        if (!(up1 > 0.0) && !(up2 > 0.0)) bad |= ST_LOAD_INVALID;
        // raise: u^i = u_i - f k_i (k.u - u_4), u^4 = -u_4 + f (k.u - u_4)
        const double kul = ku - ul4;
        const double ucov[3] = {u[0], u[1], u[2]};
        for (int q = 0; q < 3; ++q) u[q] = ucov[q] - f * kk[q] * kul;
        u[3] = -ul4 + f * kul;
      }
    } else {
      // contravariant u^i given: g_44 (u^4)^2 + 2 g_4i u^i u^4 + g_ij u^i u^j + c^2 = 0
      const double ku = kk[0] * u[0] + kk[1] * u[1] + kk[2] * u[2];
      const double A = -1.0 + f, B = 2.0 * f * ku;
      const double Cc = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + f * ku * ku + c2;
      const double disc = B * B - 4.0 * A * Cc;
      if (!(A < 0.0)) {
        bad |= ST_LOAD_ERGO;
      } else if (disc < 0.0) {
        bad |= ST_LOAD_INVALID;
      } else {
        const double sq = sqrt(disc);
        u[3] = fmax((-B + sq) / (2.0 * A), (-B - sq) / (2.0 * A));
        if (!(u[3] > 0.0)) bad |= ST_LOAD_INVALID;
      }
    }
  }
  if (bad) atomicOr(&st->flags, bad);
  for (int q = 0; q < 3; ++q) P.x[q][i] = (T)x[q];
  P.x[3][i] = (T)(x4[3 * n + i] - ct_now);
  for (int q = 0; q < 4; ++q) P.u[q][i] = (T)u[q];
  P.id[i] = ids[i];
  const int ci = min(max((int)floor(x[0]), 0), g.nx - 2);
  const int cj = min(max((int)floor(x[1]), 0), g.ny - 2);
  const int ck = min(max((int)floor(x[2]), 0), g.nz - 2);
  P.key[i] = inside ? kDead : (uint32_t)(((long long)ck * g.ny + cj) * g.nx + ci);
}

template <typename T>
__global__ void k_unload(const Particles<T> P, long long n, double* __restrict__ x4, double* __restrict__ u4,
                         uint32_t* __restrict__ ids, double ct_now) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < 3; ++q) {
    if (x4) x4[q * n + i] = (double)P.x[q][i];
  }
  if (x4) x4[3 * n + i] = (double)P.x[3][i] + ct_now;
  for (int q = 0; q < 4; ++q)
    if (u4) u4[q * n + i] = (double)P.u[q][i];
  if (ids) ids[i] = P.id[i];
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

template <typename T, bool MIXED>
void launch_push_q(const Grid& g, const Fields<T>& F, const Particles<T>& P, const Species& sp, DevStatus* st,
                   cudaStream_t stream) {
  const unsigned nb = blocks_for(P.n, 128);
  if (g.quad_order == 1)
    k_push_deposit<T, 1, MIXED><<<nb, 128, 0, stream>>>(g, F, P, sp, st);
  else if (g.quad_order == 3)
    k_push_deposit<T, 3, MIXED><<<nb, 128, 0, stream>>>(g, F, P, sp, st);
  else
    k_push_deposit<T, 2, MIXED><<<nb, 128, 0, stream>>>(g, F, P, sp, st);
}

// FP64 runs pure double; FP32 runs the mixed policy.
template <>
void launch_push_deposit<double>(const Grid& g, const Fields<double>& F, const Particles<double>& P,
                                 const Species& sp, DevStatus* st, bool, double, cudaStream_t stream) {
  if (P.n > 0) launch_push_q<double, false>(g, F, P, sp, st, stream);
}
template <>
void launch_push_deposit<float>(const Grid& g, const Fields<float>& F, const Particles<float>& P,
                                const Species& sp, DevStatus* st, bool, double, cudaStream_t stream) {
  if (P.n > 0) launch_push_q<float, true>(g, F, P, sp, st, stream);
}

template <typename T, bool MIXED>
void launch_batch_push_q(const BatchTables<T>& bt, int quad_order, cudaStream_t stream) {
  const unsigned nb = (unsigned)std::min(bt.npart, bt.persist_blocks);
  if (bt.npart == 0) return;
  if (quad_order == 1)
    k_push_deposit_batch<T, 1, MIXED><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart);
  else if (quad_order == 3)
    k_push_deposit_batch<T, 3, MIXED><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart);
  else
    k_push_deposit_batch<T, 2, MIXED><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart);
}

template <>
void launch_batch_push<double>(const BatchTables<double>& bt, int quad_order, cudaStream_t stream) {
  launch_batch_push_q<double, false>(bt, quad_order, stream);
}
template <>
void launch_batch_push<float>(const BatchTables<float>& bt, int quad_order, cudaStream_t stream) {
  launch_batch_push_q<float, true>(bt, quad_order, stream);
}

template <typename T>
void launch_load_particles(const Grid& g, const Particles<T>& P, long long n, const double* x4, const double* u4,
                           const uint32_t* ids, int umode, double ct_now, DevStatus* st, cudaStream_t stream) {
  if (n <= 0) return;
  k_load<T><<<blocks_for(n, 256), 256, 0, stream>>>(g, P, n, x4, u4, ids, umode, ct_now, st);
}

template <typename T>
void launch_unload_particles(const Particles<T>& P, long long n, double* x4, double* u4, uint32_t* ids,
                             double ct_now, cudaStream_t stream) {
  if (n <= 0) return;
  k_unload<T><<<blocks_for(n, 256), 256, 0, stream>>>(P, n, x4, u4, ids, ct_now);
}

template void launch_load_particles<float>(const Grid&, const Particles<float>&, long long, const double*,
                                           const double*, const uint32_t*, int, double, DevStatus*, cudaStream_t);
template void launch_load_particles<double>(const Grid&, const Particles<double>&, long long, const double*,
                                            const double*, const uint32_t*, int, double, DevStatus*,
                                            cudaStream_t);
template void launch_unload_particles<float>(const Particles<float>&, long long, double*, double*, uint32_t*,
                                             double, cudaStream_t);
template void launch_unload_particles<double>(const Particles<double>&, long long, double*, double*, uint32_t*,
                                              double, cudaStream_t);

}  // namespace grpic
