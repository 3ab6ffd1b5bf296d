// Field advance of the GRPIC cycle: magnetic half-step (Sec. 3.1, Eq. 10) and electric full
// step (Sec. 3.2, Eq. 12) on the staggered Yee lattice (Sec. 3, Fig. 2).
//
// Prognostic pair: covariant b = (F_yz, F_zx, F_xy) on faces, contravariant d = (F^x4, F^y4,
// F^z4) on edges.  Each update needs the other form of the tensor at its own lattice points:
//   B step:  e_i = F_i4 at the d^i edges,            then b -= (dx^4/2) curl e (forward diff.)
//   E step:  h   = F^jk at the b faces,              then d += dx^4 (4 pi/c J - div h) (backward)
// The missing components at a lattice point are the mean of the 2, 4 or 8 nearest points of
// their own lattice; the conversion uses the metric at that point (cached at create).  Each
// pass is two launches: a conversion pass into a scratch plane, then the stencil update, so
// every conversion is done once per lattice point.  Both passes stream x-fastest rows.
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

template <int TL, int SL, typename T>
__device__ __forceinline__ T avg(const T* __restrict__ a, long long c, long long sy, long long sz) {
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
      for (int dx = lx; dx <= hx; ++dx) s += __ldg(a + c + dz * sz + dy * sy + dx);
  if (cnt == 1) return s;
  return s / T(cnt);
}

// pred = true reads d from the midpoint predictor planes (time-centred E step).
template <int TL, typename T>
__device__ __forceinline__ void gather_pair(const Fields<T>& F, long long c, long long sy, long long sz, T b[3],
                                            T d[3], bool pred = false) {
  d[0] = avg<TL, 0>(pred ? F.dp[0] : F.d[0], c, sy, sz);
  d[1] = avg<TL, 1>(pred ? F.dp[1] : F.d[1], c, sy, sz);
  d[2] = avg<TL, 2>(pred ? F.dp[2] : F.d[2], c, sy, sz);
  b[0] = avg<TL, 3>(F.b[0], c, sy, sz);
  b[1] = avg<TL, 4>(F.b[1], c, sy, sz);
  b[2] = avg<TL, 5>(F.b[2], c, sy, sz);
}

template <int TL, typename T>
__device__ __forceinline__ void cached_metric(const Fields<T>& F, long long ncell, long long c, T& f, T& k0, T& k1,
                                              T& k2) {
  const T* base = F.mc + (long long)TL * 4 * ncell + c;
  f = __ldg(base);
  k0 = __ldg(base + ncell);
  k1 = __ldg(base + 2 * ncell);
  k2 = __ldg(base + 3 * ncell);
}

struct Box {
  int lo, nxb, nyb, nzb;
};

__device__ __forceinline__ bool box_cell(const Grid& g, const Box& bx, long long t, int& i, int& j, int& k) {
  const long long per = (long long)bx.nxb * bx.nyb * bx.nzb;
  if (t >= per) return false;
  if (per <= 0xffffffffll) {  // 32-bit division (a 64-bit one is a long software sequence)
    const unsigned u = (unsigned)t, r = u / (unsigned)bx.nxb;
    i = bx.lo + (int)(u - r * (unsigned)bx.nxb);
    j = bx.lo + (int)(r % (unsigned)bx.nyb);
    k = bx.lo + (int)(r / (unsigned)bx.nyb);
    return true;
  }
  i = bx.lo + (int)(t % bx.nxb);
  const long long r = t / bx.nxb;
  j = bx.lo + (int)(r % bx.nyb);
  k = bx.lo + (int)(r / bx.nyb);
  return true;
}

Box make_box(const Grid& g, int lo) {
  Box b;
  b.lo = lo;
  b.nxb = g.nx - 2 * lo;
  b.nyb = g.ny - 2 * lo;
  b.nzb = g.nz - 2 * lo;
  return b;
}

// ---- metric cache ---------------------------------------------------------------------
template <typename T>
__global__ void k_metric_cache(const Grid g, T* __restrict__ mc, uint8_t* __restrict__ mask) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int i = (int)(c % g.nx);
  const int j = (int)((c / g.nx) % g.ny);
  const int k = (int)(c / ((long long)g.nx * g.ny));
  const bool inner = i >= 2 && i <= g.nx - 3 && j >= 2 && j <= g.ny - 3 && k >= 2 && k <= g.nz - 3;
  uint8_t bits = 0;
#pragma unroll
  for (int l = 0; l < 6; ++l) {
    const double X = i + 0.5 * half(l, 0) - g.xc;
    const double Y = j + 0.5 * half(l, 1) - g.yc;
    const double Z = k + 0.5 * half(l, 2) - g.zc;
    const Kerr<double> K = kerr_eval<double>(X, Y, Z, g.m, g.a);
    const bool excised = K.flat || K.r < g.r_exc;
    const double f = excised ? 0.0 : K.f;
    mc[(l * 4 + 0) * g.ncell + c] = (T)f;
    mc[(l * 4 + 1) * g.ncell + c] = (T)K.k0;
    mc[(l * 4 + 2) * g.ncell + c] = (T)K.k1;
    mc[(l * 4 + 3) * g.ncell + c] = (T)K.k2;
    if (inner && !excised) bits |= (uint8_t)(1u << l);
  }
  mask[c] = bits;
}

// ---- per-cell stencils (shared by the single-context and the batched kernels) -------------
// covariant e_i = F_i4 at the three edge points of cell (i,j,k) into the scratch planes
template <typename T>
__device__ __forceinline__ void cov_e_cell(const Grid& g, const Fields<T>& F, int i, int j, int k) {
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  const long long c = cell_index(g, i, j, k);
  T b[3], d[3], h[3], e[3], f, k0, k1, k2;
  gather_pair<0>(F, c, sy, sz, b, d);
  cached_metric<0>(F, g.ncell, c, f, k0, k1, k2);
  contra_spatial(f, k0, k1, k2, b, d, h);
  cov_electric(f, k0, k1, k2, h, d, e);
  F.s[0][c] = e[0];
  gather_pair<1>(F, c, sy, sz, b, d);
  cached_metric<1>(F, g.ncell, c, f, k0, k1, k2);
  contra_spatial(f, k0, k1, k2, b, d, h);
  cov_electric(f, k0, k1, k2, h, d, e);
  F.s[1][c] = e[1];
  gather_pair<2>(F, c, sy, sz, b, d);
  cached_metric<2>(F, g.ncell, c, f, k0, k1, k2);
  contra_spatial(f, k0, k1, k2, b, d, h);
  cov_electric(f, k0, k1, k2, h, d, e);
  F.s[2][c] = e[2];
}

// Eq. 10 at the three face points of cell (i,j,k).  mode 0: b -= (dx4/2) curl e in place;
// 1: save b to bp, then b -= (dx4/2) curl e; 2: b = bp - dx4 curl e.  Only advanced (masked)
// locations are touched.
template <typename T>
__device__ __forceinline__ void b_update_cell(const Grid& g, const Fields<T>& F, int i, int j, int k, int mode) {
  const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
  const long long c = cell_index(g, i, j, k);
  const uint8_t bits = F.mask[c];
  const T dx4 = grid_dx4<T>(g);
  const T coef = (mode == 2) ? dx4 : dx4 * T(0.5);
  const T* ev[3] = {F.s[0], F.s[1], F.s[2]};
  // (alpha, beta) of F_{alpha beta}: b_x = F_yz, b_y = F_zx, b_z = F_xy
  const int al[3] = {1, 2, 0}, be[3] = {2, 0, 1};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (!(bits & (1u << (3 + q)))) continue;
    const T* eb = ev[be[q]];
    const T* ea = ev[al[q]];
    const T t1 = eb[c + st[al[q]]] - eb[c];
    const T t2 = -(ea[c + st[be[q]]] - ea[c]);
    const T old = (mode == 2) ? F.bp[q][c] : F.b[q][c];
    if (mode == 1) F.bp[q][c] = old;
    F.b[q][c] = old - (t1 + t2) * coef;
  }
}

// contravariant F^{jk} at the three face points of cell (i,j,k) into the scratch planes;
// pred = true takes d from the midpoint predictor
template <typename T>
__device__ __forceinline__ void contra_h_cell(const Grid& g, const Fields<T>& F, int i, int j, int k, bool pred) {
  const long long sy = g.nx, sz = (long long)g.nx * g.ny;
  const long long c = cell_index(g, i, j, k);
  T b[3], d[3], h[3], f, k0, k1, k2;
  gather_pair<3>(F, c, sy, sz, b, d, pred);
  cached_metric<3>(F, g.ncell, c, f, k0, k1, k2);
  contra_spatial(f, k0, k1, k2, b, d, h);
  F.s[0][c] = h[0];
  gather_pair<4>(F, c, sy, sz, b, d, pred);
  cached_metric<4>(F, g.ncell, c, f, k0, k1, k2);
  contra_spatial(f, k0, k1, k2, b, d, h);
  F.s[1][c] = h[1];
  gather_pair<5>(F, c, sy, sz, b, d, pred);
  cached_metric<5>(F, g.ncell, c, f, k0, k1, k2);
  contra_spatial(f, k0, k1, k2, b, d, h);
  F.s[2][c] = h[2];
}

// Eq. 12 at the three edge points of cell (i,j,k): d_out = d + coef (4 pi/c J - div h) at
// advanced locations.  predictor = true: coef = dx4/2, d_out = the predictor planes, written
// at every cell (d copied where not advanced) so they read as a whole field; otherwise
// coef = dx4 and d is updated in place.
template <typename T>
__device__ __forceinline__ void d_update_cell(const Grid& g, const Fields<T>& F, int i, int j, int k,
                                              bool predictor) {
  const long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
  const long long c = cell_index(g, i, j, k);
  const uint8_t bits = F.mask[c];
  const T dx4 = grid_dx4<T>(g);
  const T coef = predictor ? dx4 * T(0.5) : dx4;
  const T four_pi_over_c = grid_four_pi_c<T>(g);
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    T* out = predictor ? F.dp[al] : F.d[al];
    if (!(bits & (1u << al))) {
      if (predictor) out[c] = F.d[al][c];
      continue;
    }
    T div = T(0);
#pragma unroll
    for (int nu = 0; nu < 3; ++nu) {
      if (nu == al) continue;
      const int q = 3 - al - nu;  // face lattice holding F^{al nu} = +-h_q
      const int pair0 = (q == 0) ? 1 : (q == 1 ? 2 : 0);
      const T sgn = (pair0 == al) ? T(1) : T(-1);
      const T* hq = F.s[q];
      div += sgn * (hq[c] - hq[c - st[nu]]);
    }
    // FP32 fields: J rounded to FP32 with integer operations (this GPU's conversions run on its
    // reduced-rate FP64 pipe), then scaled in FP32
    T src;
    if constexpr (sizeof(T) == sizeof(float))
      src = narrow(F.J[al][c]) * four_pi_over_c;
    else
      src = four_pi_over_c * F.J[al][c];
    out[c] = F.d[al][c] + (src - div) * coef;
  }
}

// ---- single-context kernels ----------------------------------------------------------------
template <typename T>
__global__ void k_cov_e(const Grid g, const Fields<T> F, const Box bx) {
  int i, j, k;
  if (box_cell(g, bx, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) cov_e_cell(g, F, i, j, k);
}

template <typename T>
__global__ void k_b_update(const Grid g, const Fields<T> F, const Box bx, int mode) {
  int i, j, k;
  if (box_cell(g, bx, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k)) b_update_cell(g, F, i, j, k, mode);
}

template <typename T>
__global__ void k_contra_h(const Grid g, const Fields<T> F, const Box bx, bool pred) {
  int i, j, k;
  if (box_cell(g, bx, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k))
    contra_h_cell(g, F, i, j, k, pred);
}

template <typename T>
__global__ void k_d_update(const Grid g, const Fields<T> F, const Box bx, bool predictor) {
  int i, j, k;
  if (box_cell(g, bx, blockIdx.x * (long long)blockDim.x + threadIdx.x, i, j, k))
    d_update_cell(g, F, i, j, k, predictor);
}

// ---- batched kernels: grid-stride over a table of (instance, block) work items -------------
// lo = 1: conversion box [1, n-2]^3; 2: update box [2, n-3]^3; 0: the whole grid.
__device__ __forceinline__ Box box_of(const Grid& g, int lo) {
  Box b;
  b.lo = lo;
  b.nxb = g.nx - 2 * lo;
  b.nyb = g.ny - 2 * lo;
  b.nzb = g.nz - 2 * lo;
  return b;
}

// op: 0 cov_e, 1 b_update(mode), 2 contra_h(pred = mode), 3 d_update(predictor = mode),
// 4 zero J
template <typename T, int OP>
__global__ void k_batch_field(const InstDesc<T>* __restrict__ desc, const BlockEntry* __restrict__ blk, int nblk,
                              int lo, int mode) {
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    const BlockEntry e = blk[bi];
    const InstDesc<T>& D = desc[e.inst];
    const Grid& g = D.g;
    const long long t = (long long)e.block * blockDim.x + threadIdx.x;
    int i, j, k;
    if (!box_cell(g, box_of(g, lo), t, i, j, k)) continue;
    if (OP == 0) cov_e_cell(g, D.F, i, j, k);
    if (OP == 1) b_update_cell(g, D.F, i, j, k, mode);
    if (OP == 2) contra_h_cell(g, D.F, i, j, k, mode != 0);
    if (OP == 3) d_update_cell(g, D.F, i, j, k, mode != 0);
    if (OP == 4) {
      const long long c = cell_index(g, i, j, k);
      D.F.J[0][c] = 0.0;
      D.F.J[1][c] = 0.0;
      D.F.J[2][c] = 0.0;
    }
  }
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
void launch_metric_cache(const Grid& g, T* mc, uint8_t* mask, cudaStream_t st) {
  k_metric_cache<T><<<blocks_for(g.ncell, 256), 256, 0, st>>>(g, mc, mask);
}

template <typename T>
void launch_b_half(const Grid& g, const Fields<T>& F, int which, bool literal, cudaStream_t st) {
  const Box conv = make_box(g, 1), upd = make_box(g, 2);
  const long long nconv = (long long)conv.nxb * conv.nyb * conv.nzb;
  const long long nupd = (long long)upd.nxb * upd.nyb * upd.nzb;
  k_cov_e<T><<<blocks_for(nconv, 128), 128, 0, st>>>(g, F, conv);
  const int mode = literal ? 0 : (which == 0 ? 1 : 2);
  k_b_update<T><<<blocks_for(nupd, 256), 256, 0, st>>>(g, F, upd, mode);
}

template <typename T>
void launch_e_step(const Grid& g, const Fields<T>& F, bool literal, cudaStream_t st) {
  const Box conv = make_box(g, 1), upd = make_box(g, 2), all = make_box(g, 0);
  const long long nconv = (long long)conv.nxb * conv.nyb * conv.nzb;
  const long long nupd = (long long)upd.nxb * upd.nyb * upd.nzb;
  const long long nall = (long long)all.nxb * all.nyb * all.nzb;
  k_contra_h<T><<<blocks_for(nconv, 128), 128, 0, st>>>(g, F, conv, false);
  if (!literal) {
    // midpoint predictor d* = d + (dx4/2) rhs(d), then h from (b, d*)
    k_d_update<T><<<blocks_for(nall, 256), 256, 0, st>>>(g, F, all, true);
    k_contra_h<T><<<blocks_for(nconv, 128), 128, 0, st>>>(g, F, conv, true);
  }
  k_d_update<T><<<blocks_for(nupd, 256), 256, 0, st>>>(g, F, upd, false);
}

template <typename T>
void launch_batch_b_half(const BatchTables<T>& bt, int which, bool literal, cudaStream_t st) {
  const int mode = literal ? 0 : (which == 0 ? 1 : 2);
  k_batch_field<T, 0><<<std::min(bt.nconv, bt.persist_blocks), 128, 0, st>>>(bt.desc, bt.conv, bt.nconv, 1, 0);
  k_batch_field<T, 1><<<std::min(bt.nupd, bt.persist_blocks), 256, 0, st>>>(bt.desc, bt.upd, bt.nupd, 2, mode);
}

template <typename T>
void launch_batch_e_step(const BatchTables<T>& bt, bool literal, cudaStream_t st) {
  k_batch_field<T, 2><<<std::min(bt.nconv, bt.persist_blocks), 128, 0, st>>>(bt.desc, bt.conv, bt.nconv, 1, 0);
  if (!literal) {
    k_batch_field<T, 3><<<std::min(bt.nall, bt.persist_blocks), 256, 0, st>>>(bt.desc, bt.all, bt.nall, 0, 1);
    k_batch_field<T, 2><<<std::min(bt.nconv, bt.persist_blocks), 128, 0, st>>>(bt.desc, bt.conv, bt.nconv, 1, 1);
  }
  k_batch_field<T, 3><<<std::min(bt.nupd, bt.persist_blocks), 256, 0, st>>>(bt.desc, bt.upd, bt.nupd, 2, 0);
}

template <typename T>
void launch_batch_zero_j(const BatchTables<T>& bt, cudaStream_t st) {
  k_batch_field<T, 4><<<std::min(bt.nall, bt.persist_blocks), 256, 0, st>>>(bt.desc, bt.all, bt.nall, 0, 0);
}

template <typename T>
void launch_uniform_field(const Grid& g, const Fields<T>& F, const double E[3], const double B[3], cudaStream_t st) {
  k_uniform_field<T><<<blocks_for(g.ncell, 256), 256, 0, st>>>(g, F, E[0], E[1], E[2], B[0], B[1], B[2]);
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
  template void launch_metric_cache<T>(const Grid&, T*, uint8_t*, cudaStream_t);                        \
  template void launch_b_half<T>(const Grid&, const Fields<T>&, int, bool, cudaStream_t);              \
  template void launch_e_step<T>(const Grid&, const Fields<T>&, bool, cudaStream_t);                    \
  template void launch_uniform_field<T>(const Grid&, const Fields<T>&, const double*, const double*,     \
                                        cudaStream_t);                                                   \
  template void launch_convert_in<T>(T*, const double*, long long, cudaStream_t);                       \
  template void launch_convert_out<T>(double*, const T*, long long, cudaStream_t);                      \
  template void launch_batch_b_half<T>(const BatchTables<T>&, int, bool, cudaStream_t);                 \
  template void launch_batch_e_step<T>(const BatchTables<T>&, bool, cudaStream_t);                      \
  template void launch_batch_zero_j<T>(const BatchTables<T>&, cudaStream_t);

GRPIC_INST_FIELDS(float)
GRPIC_INST_FIELDS(double)

}  // namespace grpic
