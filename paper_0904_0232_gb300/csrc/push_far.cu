// FP32-mixed push with a far-field code path.  The FP32-mixed policy evaluates the quartic, the
// metric and the Christoffel contraction in FP64 wherever the FP32 estimate of r is below
// r_fp64; a particle with R(x_n) >= near_radius (common.cuh) never needs that, so it can take
// FP32-only code with no FP64 at all.  Here: the per-warp choice of code in one kernel
// (k_push_select), and the split form -- the classification of near particles for a separate
// near-hole kernel and the FP32-only push of the others (k_push_far).
#include <algorithm>
#include <cmath>

#include "push_core.cuh"

namespace grpic {

namespace {

// Mark and list the live particles with R(x_n)^2 < R_near^2.  Warp-aggregated append: the
// lanes of a warp take consecutive list slots in lane order.
template <typename T>
__global__ void k_classify_near(const Grid g, const Particles<T> P, float r_near2, uint32_t* __restrict__ list,
                                int* count) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool near = false;
  if (i < P.n && i < (long long)(*P.n_dev) && P.key[i] != kDead) {
    const float X = (float)P.x[0][i] - (float)g.xc;
    const float Y = (float)P.x[1][i] - (float)g.yc;
    const float Z = (float)P.x[2][i] - (float)g.zc;
    near = X * X + Y * Y + Z * Z < r_near2;
    if (near) P.key[i] = kNear;
  }
  const unsigned mask = __ballot_sync(0xffffffffu, near);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(count, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (near) list[base + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)i;
}

// FP32-only push of the far particles (key neither removed nor near).  MINB: resident blocks
// per SM the register allocation is sized for (4: 128 registers, 5: 96, 6: 80).
template <int Q, int MINB>
__global__ void __launch_bounds__(128, MINB) k_push_far(const Grid g, const Fields<float> F,
                                                        const Particles<float> P, const Consts<float> C,
                                                        DevStatus* st) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned flags = 0, n64 = 0;
  bool active = i < P.n && i < (long long)(*P.n_dev);
  if (active) {
    const uint32_t k = P.key[i];
    active = k != kDead && k != kNear;
  }
  if (active) push_particle<float, Q>(g, F, P, C, i, st, flags, n64, P.key + i, false);
  warp_status(st, flags, n64, active);
}

// One kernel for every particle, the policy chosen per warp: a warp none of whose particles is
// near (R(x_n) >= near_radius, the same criterion as the classification) takes the far-field
// code; a warp with any near particle takes the FP32-mixed code.  Particles are cell-sorted, so
// warps are nearly always homogeneous, and the near warps share every SM with far warps: FP64
// and FP32 work proceed side by side on their own pipes.
//
// TILE: the block accumulates J in a shared-memory FP32 tile over the nodes its particles can
// reach -- [cmin - 1, cmax + 2] per axis, cmin..cmax the cells of the block's x_n (|dx| < 1) --
// and adds the nonzero entries to the global FP64 J once at the end (one atomic per node instead
// of one per contribution).  A block whose tile would exceed kJTileFloats, and any face outside
// the tile, deposits straight to global J.
constexpr int kJTileFloats = 3072;

// perm: the block -> particle-chunk map (spread_chunk in common.cuh; 1 = in order).
// TAB: the far-field copy deposits with the per-cell area fits atab; r_near2 is then
// table_radius^2, so that every far particle lies where the fits hold.
template <int Q, int MINB, bool TILE, bool TAB = false>
__global__ void __launch_bounds__(128, MINB) k_push_select(const Grid g, const Fields<float> F,
                                                           const Particles<float> P, const Consts<float> C,
                                                           float r_near2, unsigned perm, int lg, DevStatus* st,
                                                           const float4* __restrict__ atab) {
  const unsigned chunk = spread_chunk(blockIdx.x, gridDim.x, perm, lg);
  const long long i = chunk * (long long)blockDim.x + threadIdx.x;
  unsigned flags = 0, n64 = 0;
  bool active = i < P.n && i < (long long)(*P.n_dev);
  if (active) active = P.key[i] != kDead;
  bool near = false;
  float x0[3] = {0.f, 0.f, 0.f};
  if (active) {
    x0[0] = P.x[0][i];
    x0[1] = P.x[1][i];
    x0[2] = P.x[2][i];
    const float X = x0[0] - C.xc, Y = x0[1] - C.yc, Z = x0[2] - C.zc;
    near = X * X + Y * Y + Z * Z < r_near2;
  }
  JTile jt;
  if constexpr (TILE) {
    __shared__ float s_tile[kJTileFloats];
    __shared__ int s_lo[3][4], s_hi[3][4];
    __shared__ JTile s_jt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int c = (int)floorf(x0[ax]);
      const int lo = __reduce_min_sync(0xffffffffu, active ? c : 0x7fffffff);
      const int hi = __reduce_max_sync(0xffffffffu, active ? c : -0x7fffffff);
      if (lane == 0) {
        s_lo[ax][warp] = lo;
        s_hi[ax][warp] = hi;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int lo[3], hi[3];
      for (int ax = 0; ax < 3; ++ax) {
        lo[ax] = min(min(s_lo[ax][0], s_lo[ax][1]), min(s_lo[ax][2], s_lo[ax][3]));
        hi[ax] = max(max(s_hi[ax][0], s_hi[ax][1]), max(s_hi[ax][2], s_hi[ax][3]));
      }
      JTile t;
      if (lo[0] <= hi[0]) {
        t.ox = lo[0] - 1;
        t.oy = lo[1] - 1;
        t.oz = lo[2] - 1;
        t.nx = hi[0] - lo[0] + 4;
        t.ny = hi[1] - lo[1] + 4;
        t.nz = hi[2] - lo[2] + 4;
        if ((long long)3 * t.nx * t.ny * t.nz <= kJTileFloats) t.tile = s_tile;
      }
      s_jt = t;
    }
    __syncthreads();
    jt = s_jt;
    if (jt.tile)
      for (int e = threadIdx.x; e < 3 * jt.nx * jt.ny * jt.nz; e += blockDim.x) s_tile[e] = 0.f;
    __syncthreads();
  }
  // two inlined copies, each with the flag a constant: the far-field copy has no out-of-line
  // calls at all (a call site in the loop would cost every warp registers and stack traffic)
  if (__any_sync(0xffffffffu, near)) {
    if (active) push_particle<float, Q>(g, F, P, C, i, st, flags, n64, P.key + i, true, jt);
  } else if constexpr (TAB) {
    if (active) {
      // the fits of x_n's cell (the deposit's first segment) into L2 now, read after the RK4 stages
      const int nn[3] = {g.nx, g.ny, g.nz};
      int c[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) c[ax] = min(max((int)floorf(x0[ax]), 0), nn[ax] - 2);
      const char* t = reinterpret_cast<const char*>(atab + cell_index(g, c[0], c[1], c[2]) * kAreaTableStride);
#pragma unroll
      for (int b = 0; b < 16 * kAreaTableStride; b += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(t + b));
      push_particle<float, Q, true>(g, F, P, C, i, st, flags, n64, P.key + i, false, jt, atab);
    }
  } else if (active) {
    push_particle<float, Q>(g, F, P, C, i, st, flags, n64, P.key + i, false, jt);
  }
  warp_status(st, flags, n64, active);
  if constexpr (TILE) {
    __syncthreads();
    if (jt.tile) {
      const int plane = jt.nx * jt.ny * jt.nz;
      for (int e = threadIdx.x; e < 3 * plane; e += blockDim.x) {
        const float v = jt.tile[e];
        if (v == 0.f) continue;
        const int comp = e / plane, rem = e - comp * plane;
        const int ix = jt.ox + rem % jt.nx, iy = jt.oy + (rem / jt.nx) % jt.ny, iz = jt.oz + rem / (jt.nx * jt.ny);
        if (ix < g.nx && iy < g.ny && iz < g.nz)
          atomicAdd(F.J[comp] + ((long long)iz * g.ny + iy) * g.nx + ix, widen(v));
      }
    }
  }
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_classify_near(const Grid& g, const Particles<float>& P, uint32_t* list, int* count,
                          cudaStream_t stream) {
  if (P.n <= 0) return;
  const double rn = near_radius(g);
  k_classify_near<float><<<blocks_for(P.n, 256), 256, 0, stream>>>(g, P, (float)(rn * rn), list, count);
}

int far_variant(int quad_order, int minb) {
  if (quad_order != 2) return 5;
  return (minb == 4 || minb == 6) ? minb : 5;
}

void launch_push_far(const Grid& g, const Fields<float>& F, const Particles<float>& P, const Species& sp,
                     DevStatus* st, int minb, cudaStream_t stream) {
  if (P.n <= 0) return;
  const unsigned nb = blocks_for(P.n, 128);
  const int v = far_variant(g.quad_order, minb);
  const Consts<float> C = make_consts<float>(g, sp);
  if (g.quad_order == 1)
    k_push_far<1, 5><<<nb, 128, 0, stream>>>(g, F, P, C, st);
  else if (g.quad_order == 3)
    k_push_far<3, 5><<<nb, 128, 0, stream>>>(g, F, P, C, st);
  else if (v == 4)
    k_push_far<2, 4><<<nb, 128, 0, stream>>>(g, F, P, C, st);
  else if (v == 6)
    k_push_far<2, 6><<<nb, 128, 0, stream>>>(g, F, P, C, st);
  else
    k_push_far<2, 5><<<nb, 128, 0, stream>>>(g, F, P, C, st);
}

unsigned coprime_multiplier(unsigned n) {
  // a multiplier near 0.618 n (well spread) that is coprime to n
  if (n <= 2) return 1;
  unsigned m = (unsigned)(0.6180339887 * n) | 1u;
  auto gcd = [](unsigned a, unsigned b) {
    while (b) {
      const unsigned t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  while (gcd(m, n) != 1) m += 2;
  return m % n;
}

void launch_push_select(const Grid& g, const Fields<float>& F, const Particles<float>& P, const Species& sp,
                        DevStatus* st, int minb, bool tile, int spread, const float4* atab, cudaStream_t stream) {
  if (P.n <= 0) return;
  const unsigned nb = blocks_for(P.n, 128);
  const Consts<float> C = make_consts<float>(g, sp);
  const bool tab = atab != nullptr && g.quad_order == 2 && !tile;
  const double rn = tab ? table_radius(g) : near_radius(g);
  const float r_near2 = (float)(rn * rn);
  const int lg = spread > 0 ? spread_log2(spread) : 0;
  const unsigned perm = spread > 0 ? spread_multiplier(nb, lg) : 1u;
  if (g.quad_order == 1)
    k_push_select<1, 4, false><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, nullptr);
  else if (g.quad_order == 3)
    k_push_select<3, 4, false><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, nullptr);
  else if (tab && minb >= 5)
    k_push_select<2, 5, false, true><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, atab);
  else if (tab)
    k_push_select<2, 4, false, true><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, atab);
  else if (tile && minb >= 5)
    k_push_select<2, 5, true><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, nullptr);
  else if (tile)
    k_push_select<2, 4, true><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, nullptr);
  else if (minb >= 5)
    k_push_select<2, 5, false><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, nullptr);
  else
    k_push_select<2, 4, false><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, perm, lg, st, nullptr);
}

}  // namespace grpic
