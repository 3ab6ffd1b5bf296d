// Kernels of the fused gather + GR-RK4 push + curved-metric deposit (the per-particle work is
// in push_core.cuh): the single-kernel push (FP64, and FP32-mixed without the near/far split),
// the near-hole pass of the split FP32-mixed push, the batched push, and particle load/unload.
#include <algorithm>
#include <cmath>

#include "push_core.cuh"

namespace grpic {

namespace {

template <typename T, int Q, bool MIXED>
__global__ void __launch_bounds__(128, 4) k_push_deposit(const Grid g, const Fields<T> F, const Particles<T> P,
                                                           const Consts<T> C, DevStatus* st) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned flags = 0, n64 = 0;
  bool active = i < P.n && i < (long long)(*P.n_dev);
  if (active) active = P.key[i] != kDead;
  if (active) push_particle<T, Q>(g, F, P, C, i, st, flags, n64, P.key + i, MIXED);
  warp_status(st, flags, n64, active);
}

// Block-cooperative copy of a trivially copyable struct (a multiple of 4 bytes) into shared memory.
__device__ __forceinline__ void copy_words(void* dst, const void* src, size_t bytes) {
  unsigned* d = static_cast<unsigned*>(dst);
  const unsigned* s = static_cast<const unsigned*>(src);
  for (unsigned w = threadIdx.x; w < bytes / 4; w += blockDim.x) d[w] = s[w];
}

// Near-hole pass of the split FP32-mixed push: the particles listed by the classification
// (whose stages and quadrature nodes may fall inside r < r_fp64).  Persistent blocks take
// 128-entry chunks of the list from a cursor (count[1]) until it is exhausted: the FP64 work
// per particle varies a lot, so a dynamic queue keeps the SMs evenly loaded.  Consecutive list
// entries come from consecutive cell-sorted particles, so a warp stays local.  The far kernel
// runs at the same time and tells near from far particles by the kNear mark in P.key, so the
// new sort keys go to keys[j] (by list slot) and are copied back after both end.
template <int Q>
__global__ void __launch_bounds__(128, 4) k_push_near(const Grid g, const Fields<float> F, const Particles<float> P,
                                                        const Consts<float> C, DevStatus* st,
                                                        const uint32_t* __restrict__ list, uint32_t* __restrict__ keys,
                                                        int* count) {
  __shared__ int s_base;
  const int n = count[0];
  for (;;) {
    if (threadIdx.x == 0) s_base = atomicAdd(count + 1, (int)blockDim.x);
    __syncthreads();
    const int base = s_base;
    __syncthreads();
    if (base >= n) break;
    const int j = base + threadIdx.x;
    const bool active = j < n;
    unsigned flags = 0, n64 = 0;
    if (active) push_particle<float, Q>(g, F, P, C, (long long)list[j], st, flags, n64, keys + j, true);
    warp_status(st, flags, n64, active);
  }
}

// After the join: the near particles' new sort keys back into P.key.
__global__ void k_near_keys(uint32_t* __restrict__ key, const uint32_t* __restrict__ list,
                            const uint32_t* __restrict__ keys, const int* count) {
  const int n = *count;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) key[list[j]] = keys[j];
}

// Batched: one CTA per (instance * 4 + species, block) work item; each block belongs to one
// instance and species, so the warp-level status stays per instance.  The block stages its
// instance descriptor (with the host-built launch constants) in shared memory.  The block -> item map is the same
// coprime permutation as k_push_select's (perm; 1 = in order), spreading FP64-heavy items.
// FP32-mixed: each warp takes the far-field code unless one of its particles lies within the
// instance's near_radius.
template <typename T, int Q, bool MIXED>
__global__ void __launch_bounds__(128, 4) k_push_deposit_batch(const InstDesc<T>* __restrict__ desc,
                                                                 const BlockEntry* __restrict__ blk, int nblk,
                                                                 unsigned perm) {
  __shared__ Grid sg;
  __shared__ Fields<T> sF;
  __shared__ SpeciesDesc<T> sS;
  __shared__ DevStatus* sst;
  __shared__ int s_cur;
  const int bi = (int)spread_chunk(blockIdx.x, (unsigned)nblk, perm, kBatchSpreadLog2);
  const BlockEntry e = blk[bi];
  // stage the descriptor parts this block needs with one coalesced copy by all threads (the
  // launch constants were built on the host)
  const InstDesc<T>& D = desc[e.inst >> 2];
  copy_words(&sg, &D.g, sizeof(Grid));
  copy_words(&sS, &D.sp[e.inst & 3], sizeof(SpeciesDesc<T>));
  if (threadIdx.x == 0) {
    sst = D.st;
    s_cur = *D.sp[e.inst & 3].cur;
    // the push of a batched step runs after the first B half-step: b^n is in b buffer 1
    const int dc = *D.dcur;
    for (int q = 0; q < 3; ++q) {
      sF.d[q] = D.FS.d[dc][q];
      sF.b[q] = D.FS.b[1][q];
      sF.J[q] = D.FS.J[q];
    }
  }
  __syncthreads();
  const Particles<T>& sP = sS.buf[s_cur];
  const Consts<T>& sC = sS.C;
  const float s_rnear2 = sS.r_near2;
  const long long i = (long long)e.block * blockDim.x + threadIdx.x;
  unsigned flags = 0, n64 = 0;
  bool active = i < sP.n && i < (long long)(*sP.n_dev);
  if (active) active = sP.key[i] != kDead;
  bool mixed = false;
  if constexpr (MIXED) {
    bool near = false;
    if (active) {
      const float X = sP.x[0][i] - sC.xc, Y = sP.x[1][i] - sC.yc, Z = sP.x[2][i] - sC.zc;
      near = X * X + Y * Y + Z * Z < s_rnear2;
    }
    mixed = __any_sync(0xffffffffu, near);
  }
  if (mixed) {  // two inlined copies with a constant flag (see k_push_select)
    if (active) push_particle<T, Q>(sg, sF, sP, sC, i, sst, flags, n64, sP.key + i, true);
  } else {
    if (active) push_particle<T, Q>(sg, sF, sP, sC, i, sst, flags, n64, sP.key + i, false);
  }
  warp_status(sst, flags, n64, active);
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
  const Consts<T> C = make_consts<T>(g, sp);
  if (g.quad_order == 1)
    k_push_deposit<T, 1, MIXED><<<nb, 128, 0, stream>>>(g, F, P, C, st);
  else if (g.quad_order == 3)
    k_push_deposit<T, 3, MIXED><<<nb, 128, 0, stream>>>(g, F, P, C, st);
  else
    k_push_deposit<T, 2, MIXED><<<nb, 128, 0, stream>>>(g, F, P, C, st);
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

void launch_push_near(const Grid& g, const Fields<float>& F, const Particles<float>& P, const Species& sp,
                      DevStatus* st, const uint32_t* list, uint32_t* keys, int* count, int nblocks,
                      cudaStream_t stream) {
  if (P.n <= 0 || nblocks <= 0) return;
  const Consts<float> C = make_consts<float>(g, sp);
  if (g.quad_order == 1)
    k_push_near<1><<<nblocks, 128, 0, stream>>>(g, F, P, C, st, list, keys, count);
  else if (g.quad_order == 3)
    k_push_near<3><<<nblocks, 128, 0, stream>>>(g, F, P, C, st, list, keys, count);
  else
    k_push_near<2><<<nblocks, 128, 0, stream>>>(g, F, P, C, st, list, keys, count);
}

void launch_near_keys(const Particles<float>& P, const uint32_t* list, const uint32_t* keys, const int* count,
                      int nblocks, cudaStream_t stream) {
  if (P.n <= 0 || nblocks <= 0) return;
  k_near_keys<<<nblocks, 256, 0, stream>>>(P.key, list, keys, count);
}

template <typename T, bool MIXED>
void launch_batch_push_q(const BatchTables<T>& bt, int quad_order, cudaStream_t stream) {
  // one block per work item: each block stages its instance descriptor once, and the hardware
  // scheduler balances instances of very different cost
  const unsigned nb = (unsigned)bt.npart;
  if (bt.npart == 0) return;
  const unsigned perm = spread_multiplier(nb, kBatchSpreadLog2);
  if (quad_order == 1)
    k_push_deposit_batch<T, 1, MIXED><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart, perm);
  else if (quad_order == 3)
    k_push_deposit_batch<T, 3, MIXED><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart, perm);
  else
    k_push_deposit_batch<T, 2, MIXED><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart, perm);
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
