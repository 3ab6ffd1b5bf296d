// Field advance of the GRPIC cycle: magnetic half-step (Sec. 3.1, Eq. 10) and electric full
// step (Sec. 3.2, Eq. 12) on the staggered Yee lattice (Sec. 3, Fig. 2).
//
// Prognostic pair: covariant b = (F_yz, F_zx, F_xy) on faces, contravariant d = (F^x4, F^y4,
// F^z4) on edges.  Each update needs the other form of the tensor at its own lattice points:
//   B step:  e_i = F_i4 at the d^i edges,  b_out = b_base - coef curl e(b_src, d)   (forward diff.)
//   E step:  h = F^jk at the b faces,       d_out = d + dx4 (4 pi/c J - div h)       (backward diff.)
// The missing components at a lattice point are the mean of the 2, 4 or 8 nearest points of
// their own lattice; the conversion uses the metric (f, k of Eqs. 4-6) evaluated at that point.
//
// One launch per update.  A block owns a 32 x BY patch of (x, y) columns and marches up z through
// a chunk of planes: it evaluates the conversion for the whole patch of the next plane into
// shared memory and updates the cells whose stencil lies inside the patch.  Neighbouring patches
// overlap by the stencil's reach (1 cell for the B step; 3 for the time-centred E step, whose
// midpoint predictor d* = d + (dx4/2) rhs(b, d) is converted again before the update), so each
// cell is written exactly once by one block, from inputs that no block of the launch modifies.
// The output is the other buffer of a ping-pong pair (every cell written; a copy where the
// location is not advanced), except the time-centred second B half-step, which overwrites the
// b^{n-1/2} buffer it reads only at the cell it writes.  Per cell the launch moves the
// prognostic words once: the conversions and the predictor live in registers and shared memory,
// and the metric is evaluated where it is needed instead of being read from memory.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "metric.cuh"

namespace grpic {

namespace {

// Half-cell offsets of the six field locations: 0..2 = d^x, d^y, d^z (edges),
// 3..5 = b_x, b_y, b_z (faces).
__host__ __device__ constexpr int half(int loc, int ax) {
  return (loc < 3) ? (loc == ax ? 1 : 0) : ((loc - 3) == ax ? 0 : 1);
}
// Neighbour range, along one axis, of source lattice s around a point of target lattice t.
__host__ __device__ constexpr int nb_lo(int t, int s, int ax) {
  return half(s, ax) == half(t, ax) ? 0 : (half(t, ax) == 1 ? 0 : -1);
}
__host__ __device__ constexpr int nb_hi(int t, int s, int ax) {
  return half(s, ax) == half(t, ax) ? 0 : (half(t, ax) == 1 ? 1 : 0);
}

// Reciprocal square root and reciprocal: the hardware approximations in FP32 (relative error
// ~1e-7, below the FP32 rounding of the stencil sums), IEEE operations in FP64.
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_t(double v) { return 1.0 / sqrt(v); }
__device__ __forceinline__ float rcp_t(float v) { return __fdividef(1.f, v); }
__device__ __forceinline__ double rcp_t(double v) { return 1.0 / v; }

template <typename T>
struct Pt {
  T f, k0, k1, k2;
};

// f and k of Eqs. 4-6 at location l of the cell whose lower corner is (xr, yr, zr) relative to the
// centre.  The quartic's root r^2 by the cancellation-free branch form with
// D = sqrt(p^2 + 4 a^2 z^2), p = R^2 - a^2; since the root satisfies r^4 + a^2 z^2 = r^2 (2 r^2 - p)
// = r^2 D, f = 2 m r^3 / (r^4 + a^2 z^2) = 2 m r / D.  Excised locations (and r = 0) take the flat
// metric, as the conversions there do.
template <typename T>
__device__ __forceinline__ Pt<T> metric_pt(const FieldConsts<T>& K, int l, T xr, T yr, T zr, bool excised) {
  Pt<T> P;
  P.f = T(0);
  P.k0 = T(0);
  P.k1 = T(0);
  P.k2 = T(1);
  if (excised || !K.massive) return P;
  const T X = half(l, 0) ? xr + T(0.5) : xr;
  const T Y = half(l, 1) ? yr + T(0.5) : yr;
  const T Z = half(l, 2) ? zr + T(0.5) : zr;
  const T q = K.a2 * Z * Z;
  const T p = fma(X, X, fma(Y, Y, fma(Z, Z, -K.a2)));
  const T disc = fma(p, p, T(4) * q);
  const T rD = rsqrt_t(disc);  // 1 / D
  const T D = disc * rD;
  const T r2 = p >= T(0) ? T(0.5) * (p + D) : T(2) * q * rcp_t(D - p);
  if (!(r2 > T(0))) return P;
  const T ir = rsqrt_t(r2);
  const T r = r2 * ir;
  const T irho2 = rcp_t(r2 + K.a2);
  P.f = K.two_m * r * rD;
  P.k0 = (r * X - K.a * Y) * irho2;
  P.k1 = (r * Y + K.a * X) * irho2;
  P.k2 = Z * ir;
  return P;
}

// Contravariant spatial F^{jk} from covariant b and contravariant d at one point (g = eta + f k k,
// Eq. 8): lowering gives b = M h M + f (d k^T - k d^T) with M = I + f k k^T, whose solution is
// h = [b - f (d x k) + f k (k.b)] / (1 + f) (k.(d x k) = 0 and k.k = 1, k being null for eta).
template <typename T>
__device__ __forceinline__ T h_comp(int q, const Pt<T>& P, const T b[3], T dxk_q, T inv1f) {
  const T kb = P.k0 * b[0] + P.k1 * b[1] + P.k2 * b[2];
  const T kq = q == 0 ? P.k0 : (q == 1 ? P.k1 : P.k2);
  return (b[q] - P.f * dxk_q + P.f * kq * kb) * inv1f;
}

constexpr int kTX = 32;        // threads (cells) of a patch along x: one warp per row
constexpr int kSX = kTX + 2;   // staged columns: the patch and a one-cell halo

// Three components of one z plane of a patch with a one-cell halo, staged in shared memory.
template <typename T, int BY>
struct Plane3 {
  T v[3][BY + 2][kSX];
};

// Mean of the points of source lattice SL (component SL % 3 of the staged planes S) nearest to the
// point of target lattice TL in the cell at patch position (tx, ty); the planes at z offsets -1,
// 0, +1 sit in slots sm, sc, sp.
template <int TL, int SL, typename T, int BY, int NS>
__device__ __forceinline__ T avg_s(const Plane3<T, BY> (&S)[NS], int sm, int sc, int sp, int tx, int ty) {
  constexpr int lx = nb_lo(TL, SL, 0), hx = nb_hi(TL, SL, 0);
  constexpr int ly = nb_lo(TL, SL, 1), hy = nb_hi(TL, SL, 1);
  constexpr int lz = nb_lo(TL, SL, 2), hz = nb_hi(TL, SL, 2);
  constexpr int cnt = (hx - lx + 1) * (hy - ly + 1) * (hz - lz + 1);
  T s = T(0);
#pragma unroll
  for (int dz = lz; dz <= hz; ++dz) {
    const T(&P)[BY + 2][kSX] = S[dz < 0 ? sm : (dz == 0 ? sc : sp)].v[SL % 3];
#pragma unroll
    for (int dy = ly; dy <= hy; ++dy)
#pragma unroll
      for (int dx = lx; dx <= hx; ++dx) s += P[ty + 1 + dy][tx + 1 + dx];
  }
  if (cnt == 1) return s;
  return s * (T(1) / T(cnt));
}

// Covariant e_L = F_L4 at the d^L edge of the cell at (tx, ty): all six components brought to the
// edge, h as above, then e = f (k x h) + (f - 1) d - f k (k.d).
template <int L, typename T, int BY, int NB, int ND>
__device__ __forceinline__ T edge_e(const FieldConsts<T>& K, const Plane3<T, BY> (&Sb)[NB], int bm, int bc, int bp,
                                    const Plane3<T, BY> (&Sd)[ND], int dm, int dc, int dp, int tx, int ty, T xr,
                                    T yr, T zr, bool excised) {
  T bb[3], dd[3];
  dd[0] = avg_s<L, 0>(Sd, dm, dc, dp, tx, ty);
  dd[1] = avg_s<L, 1>(Sd, dm, dc, dp, tx, ty);
  dd[2] = avg_s<L, 2>(Sd, dm, dc, dp, tx, ty);
  bb[0] = avg_s<L, 3>(Sb, bm, bc, bp, tx, ty);
  bb[1] = avg_s<L, 4>(Sb, bm, bc, bp, tx, ty);
  bb[2] = avg_s<L, 5>(Sb, bm, bc, bp, tx, ty);
  const Pt<T> P = metric_pt<T>(K, L, xr, yr, zr, excised);
  const T inv1f = rcp_t(T(1) + P.f);
  const T dxk0 = dd[1] * P.k2 - dd[2] * P.k1;
  const T dxk1 = dd[2] * P.k0 - dd[0] * P.k2;
  const T dxk2 = dd[0] * P.k1 - dd[1] * P.k0;
  const T h0 = h_comp(0, P, bb, dxk0, inv1f), h1 = h_comp(1, P, bb, dxk1, inv1f), h2 = h_comp(2, P, bb, dxk2, inv1f);
  const T kd = P.k0 * dd[0] + P.k1 * dd[1] + P.k2 * dd[2];
  T kxh, kL;
  if (L == 0) {
    kxh = P.k1 * h2 - P.k2 * h1;
    kL = P.k0;
  } else if (L == 1) {
    kxh = P.k2 * h0 - P.k0 * h2;
    kL = P.k1;
  } else {
    kxh = P.k0 * h1 - P.k1 * h0;
    kL = P.k2;
  }
  return P.f * kxh + (P.f - T(1)) * dd[L] - P.f * kL * kd;
}

// Contravariant h_Q = F^{jk} (Q = 0: F^yz, 1: F^zx, 2: F^xy) at the b_Q face of the cell at (tx, ty):
// the three b components (staged planes Sb, slots bm/bc/bp) and the two d components of (d x k)_Q
// (staged planes Sd, slots dm/dc/dp) brought to the face.
template <int Q, typename T, int BY, int NB, int ND>
__device__ __forceinline__ T face_h(const FieldConsts<T>& K, const Plane3<T, BY> (&Sb)[NB], int bm, int bc, int bp,
                                    const Plane3<T, BY> (&Sd)[ND], int dm, int dc, int dp, int tx, int ty, T xr,
                                    T yr, T zr, bool excised) {
  constexpr int L = 3 + Q;
  T bb[3];
  bb[0] = avg_s<L, 3>(Sb, bm, bc, bp, tx, ty);
  bb[1] = avg_s<L, 4>(Sb, bm, bc, bp, tx, ty);
  bb[2] = avg_s<L, 5>(Sb, bm, bc, bp, tx, ty);
  constexpr int A = (Q + 1) % 3, B = (Q + 2) % 3;  // (d x k)_Q = d_A k_B - d_B k_A
  const T dA = avg_s<L, A>(Sd, dm, dc, dp, tx, ty);
  const T dB = avg_s<L, B>(Sd, dm, dc, dp, tx, ty);
  const Pt<T> P = metric_pt<T>(K, L, xr, yr, zr, excised);
  const T kA = A == 0 ? P.k0 : (A == 1 ? P.k1 : P.k2);
  const T kB = B == 0 ? P.k0 : (B == 1 ? P.k1 : P.k2);
  return h_comp(Q, P, bb, dA * kB - dB * kA, rcp_t(T(1) + P.f));
}

// 4 pi / c J^al in the field type: FP64 J rounded to FP32 with integer operations (this GPU runs
// conversions on its reduced-rate FP64 pipe), then scaled in FP32.
template <typename T>
__device__ __forceinline__ T source(const FieldConsts<T>& K, double J) {
  if constexpr (sizeof(T) == sizeof(float))
    return narrow(J) * K.four_pi_c;
  else
    return K.four_pi_c * J;
}

__device__ __forceinline__ bool adv(uint16_t w, int l) { return (w >> l) & 1u; }
__device__ __forceinline__ bool exc(uint16_t w, int l) { return (w >> (8 + l)) & 1u; }
__device__ __forceinline__ bool in_layer(uint16_t w) { return (w & kLayerBit) != 0u; }

// ---- absorbing layers -------------------------------------------------------------------------
// Relaxation per step at location l of cell (i, j, k): the larger of the outer layer's
// k_out ((W + 1 - s) / W)^2 where s <= W, s being 1 + the cell's distance in cells to the outer two
// index layers (s = 1 at the first advanced cell), and the inner layer's
// k_in (r_abs - r) / (r_abs - r_exc) where r_exc <= r < r_abs (r at the location, in FP64).  The
// outer profile is evaluated in the field type from integers and constants converted on the host;
// the inner one is tabulated once, in FP64, over the box of cells around the hole that holds every
// location with r < r_abs, and looked up in cells flagged for it (kInnerBit).  The field kernels
// then run no FP64 operation for the layers (this GPU's FP64 pipe, which also does its
// conversions, is narrow).

// A small non-negative int as a float without a conversion instruction: the float with the bits
// of 2^23 + v, minus 2^23; exact for 0 <= v < 2^23.
__device__ __forceinline__ float small_int_to_float(int v) { return __int_as_float(0x4B000000 | v) - 8388608.f; }

template <typename T>
__device__ __forceinline__ T outer_kappa(const Grid& g, int i, int j, int k) {
  const int s = 1 + min(min(min(i - 2, g.nx - 3 - i), min(j - 2, g.ny - 3 - j)), min(k - 2, g.nz - 3 - k));
  if (s < 1 || s > g.w_out) return T(0);  // (k_out = 0 gives 0 below)
  T k_out, inv_w, n;
  if constexpr (sizeof(T) == sizeof(float)) {
    k_out = g.k_out_f;
    inv_w = g.inv_w_f;
    n = small_int_to_float(g.w_out + 1 - s);
  } else {
    k_out = g.k_out;
    inv_w = g.inv_w;
    n = (double)(g.w_out + 1 - s);
  }
  const T u = n * inv_w;
  return k_out * u * u;
}

// The inner layer's relaxation at location l of cell (i, j, k), in FP64.
__device__ inline double inner_kappa(const Grid& g, int l, int i, int j, int k) {
  if (!(g.k_in > 0.0) || !(g.r_abs > g.r_exc)) return 0.0;
  const Kerr<double> K = kerr_eval<double>(i + 0.5 * half(l, 0) - g.xc, j + 0.5 * half(l, 1) - g.yc,
                                           k + 0.5 * half(l, 2) - g.zc, g.m, g.a);
  if (K.flat || K.r < g.r_exc || K.r >= g.r_abs) return 0.0;
  return g.k_in * (g.r_abs - K.r) / (g.r_abs - g.r_exc);
}

// Index of location l of cell (i, j, k) in the inner layer's table (the cell must lie in the box).
__host__ __device__ __forceinline__ long long kin_index(const Grid& g, int l, int i, int j, int k) {
  return (((long long)l * g.kboxn[2] + (k - g.kbox0[2])) * g.kboxn[1] + (j - g.kbox0[1])) * g.kboxn[0] +
         (i - g.kbox0[0]);
}

// v relaxed toward the target t at location l of cell (i, j, k) with flags w: t + (1 - kappa)(v - t).
template <typename T>
__device__ __forceinline__ T relax(const Grid& g, const T* kin, uint16_t w, T t, T v, int l, int i, int j, int k) {
  T kap = outer_kappa<T>(g, i, j, k);
  if (w & kInnerBit) kap = fmax(kap, __ldg(kin + kin_index(g, l, i, j, k)));
  return t + (T(1) - kap) * (v - t);
}

// Asynchronous 4- or 8-byte copy global -> shared (zero-filled when ok is false: no bytes are read
// then, and src is only a valid address), and the commit / wait of the thread's copy groups.
template <typename T>
__device__ __forceinline__ void cp_async(T* dst, const T* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = ok ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's most recent copy groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The staged halo patch of a block: (BY + 2) x kSX elements, at most two per thread (threads
// 32 x BY); element e of the patch is column e % kSX, row e / kSX, at grid (x0 - 1 + column,
// y0 - 1 + row) where (x0, y0) is the grid position of thread (0, 0).
template <int BY>
struct Stager {
  int n;
  int sx[2], sy[2];
  int off[2];    // x + y nx of the element, or -1 outside the grid
  __device__ Stager(const Grid& g, int x0, int y0) {
    const int t = threadIdx.y * kTX + threadIdx.x;
    n = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = t + k * kTX * BY;
      sx[k] = sy[k] = 0;
      off[k] = -1;
      if (e < (BY + 2) * kSX) {
        n = k + 1;
        sx[k] = e % kSX;
        sy[k] = e / kSX;
        const int x = x0 - 1 + sx[k], y = y0 - 1 + sy[k];
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) off[k] = x + y * g.nx;
      }
    }
  }
  // start copying plane p of the three arrays src into dst (zeros outside the grid)
  template <typename T>
  __device__ __forceinline__ void stage(const Grid& g, const T* const* src, int p, Plane3<T, BY>& dst) const {
    const bool zin = p >= 0 && p < g.nz;
    const long long pz = zin ? (long long)p * g.nx * g.ny : 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (k < n) {
        const bool ok = zin && off[k] >= 0;
        const long long o = ok ? pz + off[k] : 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) cp_async(&dst.v[q][sy[k]][sx[k]], src[q] + o, ok);
      }
    }
  }
};

// ---- B half-step ------------------------------------------------------------------------------
// Patch: threads (tx, ty) at x = x0 + tx, y = y0 + ty; b and d of planes P-1..P+1 staged (three
// rotating slots), e at the patch of each plane P of the chunk and of the plane above it; cells
// with tx < 31 and ty < BY - 1 are updated (the curl reaches +1).
// b keeps five planes (P - 1 .. P + 1 for e, P - 1 for the update, P + 2 in flight), d four.
template <typename T, int BY>
struct BStepSmem {
  Plane3<T, BY> Sb[5], Sd[4];
  T E[2][3][BY][kTX];
};

template <typename T, int BY>
__device__ __forceinline__ void b_step_tile(const Grid& g, const BStepArgs<T>& A, int tile_x, int tile_y, int zs,
                                            int ze, BStepSmem<T, BY>& sm) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = tile_x * (kTX - 1), y0 = tile_y * (BY - 1);
  const int x = x0 + tx, y = y0 + ty;
  const bool in_xy = x < g.nx && y < g.ny;
  const bool conv_xy = x >= 1 && x <= g.nx - 2 && y >= 1 && y <= g.ny - 2;
  const bool out_xy = in_xy && tx < kTX - 1 && ty < BY - 1;
  const T xr = (T)x - A.K.xc, yr = (T)y - A.K.yc;
  const Stager<BY> st(g, x0, y0);
  auto sb = [](int p) { return (p + 5) % 5; };
  auto sd = [](int p) { return (p + 4) & 3; };
  // planes zs - 1 .. zs + 1 in one copy group; each iteration P starts plane P + 2
  for (int q = zs - 1; q <= zs + 1; ++q) {
    st.stage(g, A.src, q, sm.Sb[sb(q)]);
    st.stage(g, A.d, q, sm.Sd[sd(q)]);
  }
  cp_async_commit();
  const long long splane = (long long)g.nx * g.ny;
  uint16_t w_prev = 0;  // flags of plane P - 1, loaded one iteration ahead
  for (int P = zs; P <= ze; ++P) {
    st.stage(g, A.src, P + 2, sm.Sb[sb(P + 2)]);
    st.stage(g, A.d, P + 2, sm.Sd[sd(P + 2)]);
    cp_async_commit();
    // loads of this iteration issued ahead of the waits: the flags of plane P and, for the in-place
    // update of plane P - 1, its b^{n-1/2}
    const long long cP = ((long long)P * g.ny + y) * g.nx + x;
    const uint16_t w_cur = (in_xy && P < g.nz) ? __ldg(A.loc + cP) : (uint16_t)0;
    const int p = P - 1;
    const bool upd = p >= zs && out_xy;
    T base_old[3] = {T(0), T(0), T(0)};
    if (A.inplace && upd) {
#pragma unroll
      for (int q = 0; q < 3; ++q) base_old[q] = A.base[q][cP - splane];
    }
    cp_async_wait<1>();  // planes up to P + 1 have landed
    __syncthreads();
    // e at plane P
    {
      const int buf = P & 1;
      T e0 = T(0), e1 = T(0), e2 = T(0);
      if (conv_xy && P >= 1 && P <= g.nz - 2) {
        const uint16_t w = w_cur;
        const T zr = (T)P - A.K.zc;
        const int b0 = sb(P - 1), b1 = sb(P), b2 = sb(P + 1);
        const int d0 = sd(P - 1), d1 = sd(P), d2 = sd(P + 1);
        e0 = edge_e<0>(A.K, sm.Sb, b0, b1, b2, sm.Sd, d0, d1, d2, tx, ty, xr, yr, zr, exc(w, 0));
        e1 = edge_e<1>(A.K, sm.Sb, b0, b1, b2, sm.Sd, d0, d1, d2, tx, ty, xr, yr, zr, exc(w, 1));
        e2 = edge_e<2>(A.K, sm.Sb, b0, b1, b2, sm.Sd, d0, d1, d2, tx, ty, xr, yr, zr, exc(w, 2));
      }
      sm.E[buf][0][ty][tx] = e0;
      sm.E[buf][1][ty][tx] = e1;
      sm.E[buf][2][ty][tx] = e2;
    }
    __syncthreads();
    // b update at plane P - 1 from e of planes P - 1 and P
    if (upd) {
      const long long c = cP - splane;
      const uint16_t w = w_prev;
      const T (&E)[3][BY][kTX] = sm.E[p & 1];
      const T (&En)[3][BY][kTX] = sm.E[P & 1];
      // curl e at the three faces: b_x = F_yz: d_y e_z - d_z e_y; b_y = F_zx: d_z e_x - d_x e_z;
      // b_z = F_xy: d_x e_y - d_y e_x
      const T cx = (E[2][ty + 1][tx] - E[2][ty][tx]) - (En[1][ty][tx] - E[1][ty][tx]);
      const T cy = (En[0][ty][tx] - E[0][ty][tx]) - (E[2][ty][tx + 1] - E[2][ty][tx]);
      const T cz = (E[1][ty][tx + 1] - E[1][ty][tx]) - (E[0][ty + 1][tx] - E[0][ty][tx]);
      const T cu[3] = {cx, cy, cz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        // b at the cell: the staged b^n when the base is the source, else the other buffer
        const T old = A.inplace ? base_old[q] : sm.Sb[sb(p)].v[q][ty + 1][tx + 1];
        if (adv(w, 3 + q)) {
          T v = old - A.coef * cu[q];
          if (A.tgt[0] && in_layer(w)) v = relax<T>(g, A.kin, w, A.tgt[q][c], v, 3 + q, x, y, p);
          A.out[q][c] = v;
        } else if (!A.inplace) {
          A.out[q][c] = old;
        }
      }
    }
    w_prev = w_cur;
  }
  cp_async_wait<0>();
}

// div_al h at a cell from the face values of its plane (C) and of the plane below (M):
// F^{al nu} = +-h_q with q = 3 - al - nu, backward differences (Eq. 12):
//   div_x = (h_z - h_z[-y]) - (h_y - h_y[-z]),  div_y = (h_x - h_x[-z]) - (h_z - h_z[-x]),
//   div_z = (h_y - h_y[-x]) - (h_x - h_x[-y])
template <typename T, int BY>
__device__ __forceinline__ void div_h(const T (&C)[3][BY][kTX], const T (&M)[3][BY][kTX], int tx, int ty, T out[3]) {
  out[0] = (C[2][ty][tx] - C[2][ty - 1][tx]) - (C[1][ty][tx] - M[1][ty][tx]);
  out[1] = (C[0][ty][tx] - M[0][ty][tx]) - (C[2][ty][tx] - C[2][ty][tx - 1]);
  out[2] = (C[1][ty][tx] - C[1][ty][tx - 1]) - (C[0][ty][tx] - C[0][ty - 1][tx]);
}

// ---- E step -----------------------------------------------------------------------------------
// Patch: threads (tx, ty) at x = x0 + tx, y = y0 + ty with (x0, y0) two cells before the block's
// first output column and row.  b and d are staged plane by plane (four rotating slots each).
// Marching up z, iteration p:
//   A  h1 = h(b, d) at plane p+1, whole patch                                   [predictor only]
//   B  d* at plane p+1: d + (dx4/2)(4 pi/c J - div h1), or d where not advanced  (tx, ty >= 1)
//   C  h2 = h(b, d*) at plane p (d* at offsets 0, +1)            (1 <= tx <= 30, 1 <= ty <= BY-2)
//   D  d_out at plane p: d + dx4 (4 pi/c J - div h2)             (2 <= tx <= 30, 2 <= ty <= BY-2)
// The literal step (no predictor) skips A and takes d* = d.  The march starts 3 planes below the
// chunk, so that every buffer holds its plane when the first output plane is reached.
// b and d keep five planes each (p - 1 .. p + 2 in use, p + 3 in flight).
template <typename T, int BY>
struct EStepSmem {
  Plane3<T, BY> Sb[5], Sd[5], DP[2];
  T H1[2][3][BY][kTX];
  T H2[2][3][BY][kTX];
};

template <typename T, int BY>
__device__ __forceinline__ void e_step_tile(const Grid& g, const EStepArgs<T>& A, int tile_x, int tile_y, int zs,
                                            int ze, EStepSmem<T, BY>& sm) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = tile_x * (kTX - 3) - 2, y0 = tile_y * (BY - 3) - 2;
  const int x = x0 + tx, y = y0 + ty;
  const bool in_xy = x >= 0 && x < g.nx && y >= 0 && y < g.ny;
  const bool conv_xy = x >= 1 && x <= g.nx - 2 && y >= 1 && y <= g.ny - 2;
  const bool dp_xy = in_xy && tx >= 1 && ty >= 1;
  const bool h2_xy = conv_xy && tx >= 1 && tx <= kTX - 2 && ty >= 1 && ty <= BY - 2;
  const bool out_xy = in_xy && tx >= 2 && tx <= kTX - 2 && ty >= 2 && ty <= BY - 2;
  const T xr = (T)x - A.K.xc, yr = (T)y - A.K.yc;
  const T dx4 = A.K.dx4;
  const T half_dx4 = dx4 * T(0.5);
  const Stager<BY> st(g, x0, y0);
  auto s5 = [](int p) { return (p + 10) % 5; };
  // planes zs - 3 .. zs - 1 in one copy group; iteration p starts plane p + 3
  for (int q = zs - 3; q <= zs - 1; ++q) {
    st.stage(g, A.b, q, sm.Sb[s5(q)]);
    st.stage(g, A.d, q, sm.Sd[s5(q)]);
  }
  cp_async_commit();
  int cur = 0;  // buffer of plane p in H1, DP, H2 (plane p + 1 in the other)
  // flags and source of plane p, carried from the iteration that loaded them as plane p + 1
  uint16_t w_cur = 0;
  T src_cur[3] = {T(0), T(0), T(0)};
  const long long splane = (long long)g.nx * g.ny;
  for (int p = zs - 3; p < ze; ++p) {
    const int nxt = cur ^ 1;
    st.stage(g, A.b, p + 3, sm.Sb[s5(p + 3)]);
    st.stage(g, A.d, p + 3, sm.Sd[s5(p + 3)]);
    cp_async_commit();
    // flags and J of plane p + 1, issued ahead of the waits (J is converted where it is used)
    const int pp = p + 1;
    const bool row_in = in_xy && pp >= 0 && pp < g.nz;
    const long long cn = ((long long)pp * g.ny + y) * g.nx + x;
    const uint16_t w_next = row_in ? __ldg(A.loc + cn) : (uint16_t)0;
    double j_next[3] = {0.0, 0.0, 0.0};
    if (row_in) {
#pragma unroll
      for (int al = 0; al < 3; ++al) j_next[al] = __ldg(A.J[al] + cn);
    }
    cp_async_wait<1>();  // planes up to p + 2 have landed
    __syncthreads();
    // A: h1 at plane p + 1
    if (A.pred) {
      T v0 = T(0), v1 = T(0), v2 = T(0);
      const int pp = p + 1;
      if (conv_xy && pp >= 1 && pp <= g.nz - 2) {
        const uint16_t w = w_next;
        const T zr = (T)pp - A.K.zc;
        const int a = s5(p), b = s5(p + 1), d = s5(p + 2);
        v0 = face_h<0>(A.K, sm.Sb, a, b, d, sm.Sd, a, b, d, tx, ty, xr, yr, zr, exc(w, 3));
        v1 = face_h<1>(A.K, sm.Sb, a, b, d, sm.Sd, a, b, d, tx, ty, xr, yr, zr, exc(w, 4));
        v2 = face_h<2>(A.K, sm.Sb, a, b, d, sm.Sd, a, b, d, tx, ty, xr, yr, zr, exc(w, 5));
      }
      sm.H1[nxt][0][ty][tx] = v0;
      sm.H1[nxt][1][ty][tx] = v1;
      sm.H1[nxt][2][ty][tx] = v2;
    }
    __syncthreads();
    // B: d* at plane p + 1
    T src_next[3];
#pragma unroll
    for (int al = 0; al < 3; ++al) src_next[al] = source<T>(A.K, j_next[al]);
    {
      if (dp_xy && pp >= 0 && pp < g.nz && p >= zs - 2) {
        const Plane3<T, BY>& Dn = sm.Sd[s5(pp)];
        T dv[3] = {Dn.v[0][ty + 1][tx + 1], Dn.v[1][ty + 1][tx + 1], Dn.v[2][ty + 1][tx + 1]};
        if (A.pred) {
          T dv_h[3];
          div_h<T, BY>(sm.H1[nxt], sm.H1[cur], tx, ty, dv_h);
#pragma unroll
          for (int al = 0; al < 3; ++al)
            if (adv(w_next, al)) dv[al] += (src_next[al] - dv_h[al]) * half_dx4;
        }
        sm.DP[nxt].v[0][ty + 1][tx + 1] = dv[0];
        sm.DP[nxt].v[1][ty + 1][tx + 1] = dv[1];
        sm.DP[nxt].v[2][ty + 1][tx + 1] = dv[2];
      }
    }
    __syncthreads();
    // C: h2 = h(b, d*) at plane p (d* of planes p and p + 1 in DP[cur], DP[nxt])
    if (p >= zs - 1) {
      T v0 = T(0), v1 = T(0), v2 = T(0);
      if (h2_xy && p >= 1 && p <= g.nz - 2) {
        const uint16_t w = w_cur;
        const T zr = (T)p - A.K.zc;
        const int a = s5(p - 1), b = s5(p), d = s5(p + 1);
        v0 = face_h<0>(A.K, sm.Sb, a, b, d, sm.DP, nxt, cur, nxt, tx, ty, xr, yr, zr, exc(w, 3));
        v1 = face_h<1>(A.K, sm.Sb, a, b, d, sm.DP, nxt, cur, nxt, tx, ty, xr, yr, zr, exc(w, 4));
        v2 = face_h<2>(A.K, sm.Sb, a, b, d, sm.DP, nxt, cur, nxt, tx, ty, xr, yr, zr, exc(w, 5));
      }
      sm.H2[cur][0][ty][tx] = v0;
      sm.H2[cur][1][ty][tx] = v1;
      sm.H2[cur][2][ty][tx] = v2;
    }
    __syncthreads();
    // D: d_out at plane p (h2 of plane p in H2[cur], of plane p - 1 in H2[nxt])
    if (p >= zs && out_xy) {
      const long long c = cn - splane;
      const Plane3<T, BY>& Dc = sm.Sd[s5(p)];
      T dv_h[3];
      div_h<T, BY>(sm.H2[cur], sm.H2[nxt], tx, ty, dv_h);
#pragma unroll
      T v[3];
#pragma unroll
      for (int al = 0; al < 3; ++al) {
        const T dold = Dc.v[al][ty + 1][tx + 1];
        v[al] = adv(w_cur, al) ? dold + (src_cur[al] - dv_h[al]) * dx4 : dold;
      }
      if (A.tgt[0] && in_layer(w_cur)) {
        for (int al = 0; al < 3; ++al)
          if (adv(w_cur, al)) v[al] = relax<T>(g, A.kin, w_cur, A.tgt[al][c], v[al], al, x, y, p);
      }
#pragma unroll
      for (int al = 0; al < 3; ++al) A.out[al][c] = v[al];
    }
    cur = nxt;
    w_cur = w_next;
#pragma unroll
    for (int al = 0; al < 3; ++al) src_cur[al] = src_next[al];
  }
  cp_async_wait<0>();
}

// Rows of a patch: FP32 16, FP64 8.
template <typename T>
constexpr int patch_rows() {
  return sizeof(T) == sizeof(float) ? 16 : 8;
}

// Patches of a grid for the B step (out = 31 x (BY - 1) cells) or the E step (29 x (BY - 3)), and the
// z chunk (4 to 64 planes) that minimises the estimated time: a chunk marches `halo` planes beyond
// its own and the busiest of the `sms` multiprocessors runs ceil(patches / sms) of them.
TileGrid tile_grid(const Grid& g, bool e_step, int rows, int sms) {
  TileGrid t;
  const int ox = e_step ? kTX - 3 : kTX - 1, oy = e_step ? rows - 3 : rows - 1;
  const int halo = e_step ? 4 : 2;  // planes marched (and staged) below and above the chunk
  t.ntx = (g.nx + ox - 1) / ox;
  t.nty = (g.ny + oy - 1) / oy;
  double best = 1e300;
  for (int zc = 64; zc >= 4; zc /= 2) {
    const long long nt = (long long)t.ntx * t.nty * ((g.nz + zc - 1) / zc);
    const double per_sm = std::ceil((double)nt / sms);
    const double cost = per_sm * (zc + halo);  // time ~ blocks of the busiest SM x planes marched
    if (cost < best * 0.999) {
      best = cost;
      t.zchunk = zc;
    }
  }
  t.ntz = (g.nz + t.zchunk - 1) / t.zchunk;
  return t;
}

__device__ __forceinline__ void decode_tile(const TileGrid& t, long long q, int& tx, int& ty, int& zs) {
  tx = (int)(q % t.ntx);
  const long long r = q / t.ntx;
  ty = (int)(r % t.nty);
  zs = (int)(r / t.nty) * t.zchunk;
}

template <typename T, int BY>
__global__ void __launch_bounds__(kTX * BY, 2) k_b_step(const Grid g, const BStepArgs<T> A, const TileGrid t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<BStepSmem<T, BY>*>(smem_raw);
  int tx, ty, zs;
  decode_tile(t, blockIdx.x, tx, ty, zs);
  b_step_tile<T, BY>(g, A, tx, ty, zs, min(zs + t.zchunk, g.nz), sm);
}

template <typename T, int BY>
__global__ void __launch_bounds__(kTX * BY, 2) k_e_step(const Grid g, const EStepArgs<T> A, const TileGrid t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<EStepSmem<T, BY>*>(smem_raw);
  int tx, ty, zs;
  decode_tile(t, blockIdx.x, tx, ty, zs);
  e_step_tile<T, BY>(g, A, tx, ty, zs, min(zs + t.zchunk, g.nz), sm);
}

// ---- batched: persistent grid-stride over a table of (instance, patch) work items --------------
// which: 0 first B half (b[0] -> b[1]), 1 second B half, 2 E step.  The instance's d buffer
// parity is read from the device (flipped by launch_batch_flip_d at the end of a step).
template <typename T>
__device__ __forceinline__ const FieldConsts<T>& inst_consts(const InstDesc<T>& D) {
  if constexpr (sizeof(T) == sizeof(float))
    return D.K32;
  else
    return D.K64;
}

template <typename T>
__device__ __forceinline__ BStepArgs<T> batch_b_args(const InstDesc<T>& D, int which, bool literal) {
  BStepArgs<T> A;
  const int dc = *D.dcur;
  A.K = inst_consts(D);
  const T dx4 = A.K.dx4;
  for (int q = 0; q < 3; ++q) {
    A.d[q] = D.FS.d[dc][q];
    if (which == 0) {
      A.src[q] = D.FS.b[0][q];
      A.base[q] = D.FS.b[0][q];
      A.out[q] = D.FS.b[1][q];
    } else {
      A.src[q] = D.FS.b[1][q];
      A.base[q] = literal ? D.FS.b[1][q] : D.FS.b[0][q];
      A.out[q] = D.FS.b[0][q];
    }
  }
  for (int q = 0; q < 3; ++q) A.tgt[q] = which == 1 ? D.FS.tgt[3 + q] : nullptr;
  A.kin = D.FS.kin;
  A.loc = D.FS.loc;
  A.coef = (which == 1 && !literal) ? dx4 : dx4 * T(0.5);
  A.inplace = which == 1 && !literal;
  return A;
}

template <typename T>
__device__ __forceinline__ EStepArgs<T> batch_e_args(const InstDesc<T>& D, bool literal) {
  EStepArgs<T> A;
  const int dc = *D.dcur;
  A.K = inst_consts(D);
  for (int q = 0; q < 3; ++q) {
    A.b[q] = D.FS.b[0][q];
    A.d[q] = D.FS.d[dc][q];
    A.out[q] = D.FS.d[dc ^ 1][q];
    A.J[q] = D.FS.J[q];
    A.tgt[q] = D.FS.tgt[q];
  }
  A.kin = D.FS.kin;
  A.loc = D.FS.loc;
  A.pred = !literal;
  return A;
}

template <typename T, int BY>
__global__ void __launch_bounds__(kTX * BY) k_batch_b_step(const InstDesc<T>* __restrict__ desc,
                                                           const BlockEntry* __restrict__ blk, int nblk, int which,
                                                           bool literal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<BStepSmem<T, BY>*>(smem_raw);
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    const BlockEntry e = blk[bi];
    const InstDesc<T>& D = desc[e.inst];
    int tx, ty, zs;
    decode_tile(D.btiles, e.block, tx, ty, zs);
    b_step_tile<T, BY>(D.g, batch_b_args(D, which, literal), tx, ty, zs, min(zs + D.btiles.zchunk, D.g.nz), sm);
    __syncthreads();  // the next item restages the planes
  }
}

template <typename T, int BY>
__global__ void __launch_bounds__(kTX * BY) k_batch_e_step(const InstDesc<T>* __restrict__ desc,
                                                           const BlockEntry* __restrict__ blk, int nblk, bool literal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<EStepSmem<T, BY>*>(smem_raw);
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    const BlockEntry e = blk[bi];
    const InstDesc<T>& D = desc[e.inst];
    int tx, ty, zs;
    decode_tile(D.etiles, e.block, tx, ty, zs);
    e_step_tile<T, BY>(D.g, batch_e_args(D, literal), tx, ty, zs, min(zs + D.etiles.zchunk, D.g.nz), sm);
    __syncthreads();
  }
}

template <typename T>
__global__ void k_batch_zero_j(const InstDesc<T>* __restrict__ desc, const BlockEntry* __restrict__ blk, int nblk) {
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    const BlockEntry e = blk[bi];
    const InstDesc<T>& D = desc[e.inst];
    const long long c = (long long)e.block * blockDim.x + threadIdx.x;
    if (c < D.g.ncell) {
      D.FS.J[0][c] = 0.0;
      D.FS.J[1][c] = 0.0;
      D.FS.J[2][c] = 0.0;
    }
  }
}

template <typename T>
__global__ void k_batch_flip_d(const InstDesc<T>* __restrict__ desc, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) *desc[i].dcur ^= 1;
}

// ---- location flags --------------------------------------------------------------------------
// bit l: location l of the cell is advanced (cell in [2, n-3]^3 and r >= r_excise); bit 6: an
// advanced location of the cell has a relaxation kappa > 0; bit 7: one from the inner layer;
// bit 8 + l: location l is excised
// (r < r_excise, or r = 0), where conversions take the flat metric.  Decided once, in FP64.
__global__ void k_location_flags(const Grid g, uint16_t* __restrict__ loc) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int i = (int)(c % g.nx);
  const int j = (int)((c / g.nx) % g.ny);
  const int k = (int)(c / ((long long)g.nx * g.ny));
  const bool inner = i >= 2 && i <= g.nx - 3 && j >= 2 && j <= g.ny - 3 && k >= 2 && k <= g.nz - 3;
  unsigned w = 0;
#pragma unroll
  for (int l = 0; l < 6; ++l) {
    const double X = i + 0.5 * half(l, 0) - g.xc;
    const double Y = j + 0.5 * half(l, 1) - g.yc;
    const double Z = k + 0.5 * half(l, 2) - g.zc;
    const Kerr<double> K = kerr_eval<double>(X, Y, Z, g.m, g.a);
    const bool excised = K.flat || K.r < g.r_exc;
    if (excised) w |= 1u << (8 + l);
    if (inner && !excised) {
      w |= 1u << l;
      if (outer_kappa<double>(g, i, j, k) > 0.0) w |= kLayerBit;
      // (the box holds every such cell by construction; checked so that no lookup can leave it)
      const bool in_box = i >= g.kbox0[0] && i < g.kbox0[0] + g.kboxn[0] && j >= g.kbox0[1] &&
                          j < g.kbox0[1] + g.kboxn[1] && k >= g.kbox0[2] && k < g.kbox0[2] + g.kboxn[2];
      if (in_box && inner_kappa(g, l, i, j, k) > 0.0) w |= kLayerBit | kInnerBit;
    }
  }
  loc[c] = (uint16_t)w;
}

// ---- initial conditions / conversions ----------------------------------------------------
template <typename T>
__global__ void k_uniform_field(const Grid g, const Fields<T> F, double E0, double E1, double E2, double B0,
                                double B1, double B2) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int i = (int)(c % g.nx);
  const int j = (int)((c / g.nx) % g.ny);
  const int k = (int)(c / ((long long)g.nx * g.ny));
  const double h[3] = {B0, B1, B2};
  const double d[3] = {-E0, -E1, -E2};
  F.d[0][c] = (T)d[0];
  F.d[1][c] = (T)d[1];
  F.d[2][c] = (T)d[2];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int l = 3 + q;
    const double X = i + 0.5 * half(l, 0) - g.xc;
    const double Y = j + 0.5 * half(l, 1) - g.yc;
    const double Z = k + 0.5 * half(l, 2) - g.zc;
    const Kerr<double> K = kerr_eval<double>(X, Y, Z, g.m, g.a);
    const bool excised = K.flat || K.r < g.r_exc;
    double bl[3];
    lower_spatial<double>(excised ? 0.0 : K.f, K.k0, K.k1, K.k2, h, d, bl);
    F.b[q][c] = (T)bl[q];
  }
}

// ---- read-out of the contravariant face components --------------------------------------------
// Mean of the points of source lattice SL nearest to the point of target lattice TL in cell
// (i, j, k), from global memory, in the order of avg_s.
template <int TL, int SL, typename T>
__device__ __forceinline__ T avg_g(const T* __restrict__ F, const Grid& g, int i, int j, int k) {
  constexpr int lx = nb_lo(TL, SL, 0), hx = nb_hi(TL, SL, 0);
  constexpr int ly = nb_lo(TL, SL, 1), hy = nb_hi(TL, SL, 1);
  constexpr int lz = nb_lo(TL, SL, 2), hz = nb_hi(TL, SL, 2);
  constexpr int cnt = (hx - lx + 1) * (hy - ly + 1) * (hz - lz + 1);
  T s = T(0);
#pragma unroll
  for (int dz = lz; dz <= hz; ++dz)
#pragma unroll
    for (int dy = ly; dy <= hy; ++dy)
#pragma unroll
      for (int dx = lx; dx <= hx; ++dx) s += F[((long long)(k + dz) * g.ny + (j + dy)) * g.nx + (i + dx)];
  if (cnt == 1) return s;
  return s * (T(1) / T(cnt));
}

template <int Q, typename T>
__device__ __forceinline__ double face_h_g(const Grid& g, const FieldConsts<T>& K, const Fields<T>& F, int i, int j,
                                           int k, bool excised) {
  constexpr int L = 3 + Q;
  T bb[3];
  bb[0] = avg_g<L, 3>(F.b[0], g, i, j, k);
  bb[1] = avg_g<L, 4>(F.b[1], g, i, j, k);
  bb[2] = avg_g<L, 5>(F.b[2], g, i, j, k);
  constexpr int A = (Q + 1) % 3, B = (Q + 2) % 3;  // (d x k)_Q = d_A k_B - d_B k_A
  const T dA = avg_g<L, A>(F.d[A], g, i, j, k);
  const T dB = avg_g<L, B>(F.d[B], g, i, j, k);
  const Pt<T> P = metric_pt<T>(K, L, (T)i - K.xc, (T)j - K.yc, (T)k - K.zc, excised);
  const T kA = A == 0 ? P.k0 : (A == 1 ? P.k1 : P.k2);
  const T kB = B == 0 ? P.k0 : (B == 1 ? P.k1 : P.k2);
  return (double)h_comp(Q, P, bb, dA * kB - dB * kA, rcp_t(T(1) + P.f));
}

// h (F^yz, F^zx, F^xy) at every b face of the cells 1 .. n-2 per axis, as the E step converts the
// field; zero on the outer index layer.
template <typename T>
__global__ void k_contra_h(const Grid g, const FieldConsts<T> K, const Fields<T> F, const uint16_t* __restrict__ loc,
                           double* __restrict__ h0, double* __restrict__ h1, double* __restrict__ h2) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int i = (int)(c % g.nx);
  const int j = (int)((c / g.nx) % g.ny);
  const int k = (int)(c / ((long long)g.nx * g.ny));
  if (i < 1 || j < 1 || k < 1 || i > g.nx - 2 || j > g.ny - 2 || k > g.nz - 2) {
    h0[c] = h1[c] = h2[c] = 0.0;
    return;
  }
  const uint16_t w = loc[c];
  h0[c] = face_h_g<0, T>(g, K, F, i, j, k, exc(w, 3));
  h1[c] = face_h_g<1, T>(g, K, F, i, j, k, exc(w, 4));
  h2[c] = face_h_g<2, T>(g, K, F, i, j, k, exc(w, 5));
}

template <typename T>
__global__ void k_convert_in(T* __restrict__ dst, const double* __restrict__ src, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)src[i];
}
template <typename T>
__global__ void k_convert_out(double* __restrict__ dst, const T* __restrict__ src, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

template <typename T>
void launch_contra_h(const Grid& g, const Fields<T>& F, const uint16_t* loc, double* h3, cudaStream_t st) {
  k_contra_h<T><<<blocks_for(g.ncell, 256), 256, 0, st>>>(g, field_consts<T>(g), F, loc, h3, h3 + g.ncell,
                                                   h3 + 2 * g.ncell);
}
template void launch_contra_h<float>(const Grid&, const Fields<float>&, const uint16_t*, double*, cudaStream_t);
template void launch_contra_h<double>(const Grid&, const Fields<double>&, const uint16_t*, double*, cudaStream_t);

void launch_location_flags(const Grid& g, uint16_t* loc, cudaStream_t st) {
  k_location_flags<<<blocks_for(g.ncell, 256), 256, 0, st>>>(g, loc);
}

template <typename T>
__global__ void k_inner_kappa_table(const Grid g, T* __restrict__ kin, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int i = g.kbox0[0] + (int)(e % g.kboxn[0]);
  long long r = e / g.kboxn[0];
  const int j = g.kbox0[1] + (int)(r % g.kboxn[1]);
  r /= g.kboxn[1];
  const int k = g.kbox0[2] + (int)(r % g.kboxn[2]);
  const int l = (int)(r / g.kboxn[2]);
  kin[e] = (T)inner_kappa(g, l, i, j, k);
}

template <typename T>
void launch_inner_kappa_table(const Grid& g, T* kin, cudaStream_t st) {
  const long long n = 6ll * g.kboxn[0] * g.kboxn[1] * g.kboxn[2];
  if (n > 0) k_inner_kappa_table<T><<<blocks_for(n, 256), 256, 0, st>>>(g, kin, n);
}
template void launch_inner_kappa_table<float>(const Grid&, float*, cudaStream_t);
template void launch_inner_kappa_table<double>(const Grid&, double*, cudaStream_t);

// Dynamic shared memory of the field kernels (above the 48 KB default): set once per kernel.
template <typename K>
void allow_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
void launch_b_step(const Grid& g, const BStepArgs<T>& A, int sms, cudaStream_t st) {
  constexpr int BY = patch_rows<T>();
  constexpr size_t smem = sizeof(BStepSmem<T, BY>);
  static bool once = (allow_smem(k_b_step<T, BY>, smem), true);
  (void)once;
  const TileGrid t = tile_grid(g, false, BY, sms);
  k_b_step<T, BY><<<(unsigned)t.count(), dim3(kTX, BY), smem, st>>>(g, A, t);
}

template <typename T>
void launch_e_step(const Grid& g, const EStepArgs<T>& A, int sms, cudaStream_t st) {
  constexpr int BY = patch_rows<T>();
  constexpr size_t smem = sizeof(EStepSmem<T, BY>);
  static bool once = (allow_smem(k_e_step<T, BY>, smem), true);
  (void)once;
  const TileGrid t = tile_grid(g, true, BY, sms);
  k_e_step<T, BY><<<(unsigned)t.count(), dim3(kTX, BY), smem, st>>>(g, A, t);
}

// Patch tables of an instance for the batched field launches: z chunks of 16 planes, the
// instances themselves supplying the parallelism.
void batch_field_tiles(const Grid& g, bool fp32, TileGrid* btiles, TileGrid* etiles) {
  const int rows = fp32 ? patch_rows<float>() : patch_rows<double>();
  for (int e = 0; e < 2; ++e) {
    TileGrid t = tile_grid(g, e == 1, rows, 1);
    t.zchunk = 16;
    t.ntz = (g.nz + 15) / 16;
    *(e ? etiles : btiles) = t;
  }
}

template <typename T>
void launch_batch_b_half(const BatchTables<T>& bt, int which, bool literal, cudaStream_t st) {
  constexpr int BY = patch_rows<T>();
  constexpr size_t smem = sizeof(BStepSmem<T, BY>);
  static bool once = (allow_smem(k_batch_b_step<T, BY>, smem), true);
  (void)once;
  if (bt.nbtile == 0) return;
  k_batch_b_step<T, BY><<<std::min(bt.nbtile, bt.persist_field_blocks), dim3(kTX, BY), smem, st>>>(
      bt.desc, bt.btile, bt.nbtile, which, literal);
}

template <typename T>
void launch_batch_e_step(const BatchTables<T>& bt, bool literal, cudaStream_t st) {
  constexpr int BY = patch_rows<T>();
  constexpr size_t smem = sizeof(EStepSmem<T, BY>);
  static bool once = (allow_smem(k_batch_e_step<T, BY>, smem), true);
  (void)once;
  if (bt.netile == 0) return;
  k_batch_e_step<T, BY><<<std::min(bt.netile, bt.persist_field_blocks), dim3(kTX, BY), smem, st>>>(
      bt.desc, bt.etile, bt.netile, literal);
}

template <typename T>
void launch_batch_zero_j(const BatchTables<T>& bt, cudaStream_t st) {
  k_batch_zero_j<T><<<std::min(bt.nall, bt.persist_blocks), 256, 0, st>>>(bt.desc, bt.all, bt.nall);
}

template <typename T>
void launch_batch_flip_d(const BatchTables<T>& bt, int ninst, cudaStream_t st) {
  k_batch_flip_d<T><<<(ninst + 127) / 128, 128, 0, st>>>(bt.desc, ninst);
}

template <typename T>
void launch_uniform_field(const Grid& g, const Fields<T>& F, const double E[3], const double B[3], cudaStream_t st) {
  k_uniform_field<T><<<blocks_for(g.ncell, 256), 256, 0, st>>>(g, F, E[0], E[1], E[2], B[0], B[1], B[2]);
}

__global__ void k_add_f64(double* __restrict__ dst, const double* __restrict__ src, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] += src[i];
}

void launch_add_f64(double* dst, const double* src, long long n, cudaStream_t st) {
  if (n > 0) k_add_f64<<<blocks_for(n, 256), 256, 0, st>>>(dst, src, n);
}

template <typename T>
void launch_convert_in(T* dst, const double* src, long long n, cudaStream_t st) {
  k_convert_in<T><<<blocks_for(n, 256), 256, 0, st>>>(dst, src, n);
}
template <typename T>
void launch_convert_out(double* dst, const T* src, long long n, cudaStream_t st) {
  k_convert_out<T><<<blocks_for(n, 256), 256, 0, st>>>(dst, src, n);
}

#define GRPIC_INST_FIELDS(T)                                                                             \
  template void launch_b_step<T>(const Grid&, const BStepArgs<T>&, int, cudaStream_t);                  \
  template void launch_e_step<T>(const Grid&, const EStepArgs<T>&, int, cudaStream_t);                  \
  template void launch_uniform_field<T>(const Grid&, const Fields<T>&, const double*, const double*,     \
                                        cudaStream_t);                                                   \
  template void launch_convert_in<T>(T*, const double*, long long, cudaStream_t);                       \
  template void launch_convert_out<T>(double*, const T*, long long, cudaStream_t);                      \
  template void launch_batch_b_half<T>(const BatchTables<T>&, int, bool, cudaStream_t);                 \
  template void launch_batch_e_step<T>(const BatchTables<T>&, bool, cudaStream_t);                      \
  template void launch_batch_zero_j<T>(const BatchTables<T>&, cudaStream_t);                            \
  template void launch_batch_flip_d<T>(const BatchTables<T>&, int, cudaStream_t);

GRPIC_INST_FIELDS(float)
GRPIC_INST_FIELDS(double)

}  // namespace grpic
