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
template <int Q, int MINB>
__global__ void __launch_bounds__(128, MINB) k_push_select(const Grid g, const Fields<float> F,
                                                           const Particles<float> P, const Consts<float> C,
                                                           float r_near2, DevStatus* st) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned flags = 0, n64 = 0;
  bool active = i < P.n && i < (long long)(*P.n_dev);
  if (active) active = P.key[i] != kDead;
  bool near = false;
  if (active) {
    const float X = P.x[0][i] - C.xc, Y = P.x[1][i] - C.yc, Z = P.x[2][i] - C.zc;
    near = X * X + Y * Y + Z * Z < r_near2;
  }
  // two inlined copies, each with the flag a constant: the far-field copy has no out-of-line
  // calls at all (a call site in the loop would cost every warp registers and stack traffic)
  if (__any_sync(0xffffffffu, near)) {
    if (active) push_particle<float, Q>(g, F, P, C, i, st, flags, n64, P.key + i, true);
  } else {
    if (active) push_particle<float, Q>(g, F, P, C, i, st, flags, n64, P.key + i, false);
  }
  warp_status(st, flags, n64, active);
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

void launch_push_select(const Grid& g, const Fields<float>& F, const Particles<float>& P, const Species& sp,
                        DevStatus* st, int minb, cudaStream_t stream) {
  if (P.n <= 0) return;
  const unsigned nb = blocks_for(P.n, 128);
  const Consts<float> C = make_consts<float>(g, sp);
  const double rn = near_radius(g);
  const float r_near2 = (float)(rn * rn);
  if (g.quad_order == 1)
    k_push_select<1, 4><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, st);
  else if (g.quad_order == 3)
    k_push_select<3, 4><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, st);
  else if (minb >= 5)
    k_push_select<2, 5><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, st);
  else
    k_push_select<2, 4><<<nb, 128, 0, stream>>>(g, F, P, C, r_near2, st);
}

}  // namespace grpic
