// Diagnostics of the current: charge density at the nodes and the Gauss-law residual.
//
// rho (or J^4 / c with gamma): cloud-in-cell charge of each particle at the 8 nodes around it,
// weights trilinear in the position (the sqrt(-det g) sub-volumes of Sec. 3.3 reduce to that, det g
// being -1), times gamma = u^4 / c for the time component of J = rho gamma v (Sec. 4).
// Gauss residual at node (i, j, k): div E - 4 pi rho with E^a = -d^a = -F^{a4} and backward
// differences of the edge-centred d (the node's own edge minus the one below it on each axis),
// the discrete divergence that the E step (Eq. 12) and the zig-zag deposit keep consistent: with
// the gamma-free deposit in flat space it changes per step by exactly -4 pi times the deposit's
// 3-D continuity defect.
//
// Invariants of each particle's motion: the normalisation g_mn u^m u^n = -c^2 (Eq. 7), kept by the
// exact dynamics in any field (F is antisymmetric), and the Killing energy E = -u_4 and axial
// momentum L = u_phi = x u_y - y u_x (covariant components, position from the centre), kept along
// field-free orbits (the metric is stationary and axisymmetric; Eq. 3).  Evaluated in FP64 from the
// stored state.
#include <cmath>

#include "common.cuh"
#include "metric.cuh"

namespace grpic {

namespace {

template <typename T>
__global__ void k_charge_density(const Particles<T> P, double q, int nx, int ny, int nz, double inv_c,
                                 bool with_gamma, double* __restrict__ rho) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= P.n || i >= (long long)(*P.n_dev) || P.key[i] == kDead) return;
  const double x = (double)P.x[0][i], y = (double)P.x[1][i], z = (double)P.x[2][i];
  const int i0 = min(max((int)floor(x), 0), nx - 2), j0 = min(max((int)floor(y), 0), ny - 2);
  const int k0 = min(max((int)floor(z), 0), nz - 2);
  const double wx = x - i0, wy = y - j0, wz = z - k0;
  const double qq = with_gamma ? q * (double)P.u[3][i] * inv_c : q;
  const long long base = ((long long)k0 * ny + j0) * nx + i0;
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const double W = (di ? wx : 1.0 - wx) * (dj ? wy : 1.0 - wy) * (dk ? wz : 1.0 - wz);
        atomicAdd(rho + base + (long long)dk * nx * ny + dj * nx + di, qq * W);
      }
}

// res = div E - 4 pi rho; the max of |res| over nodes [lo, n - 1 - lo]^3 goes to *maxabs
// (atomicMax on the bit pattern of the non-negative double).
template <typename T>
__global__ void k_gauss(const T* __restrict__ dx, const T* __restrict__ dy, const T* __restrict__ dz,
                        const double* __restrict__ rho, int nx, int ny, int nz, int lo, double* __restrict__ res,
                        unsigned long long* maxabs) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ncell = (long long)nx * ny * nz;
  double worst = 0.0;
  if (idx < ncell) {
    const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((long long)nx * ny));
    double div = 0.0;
    if (i > 0) div -= (double)dx[idx] - (double)dx[idx - 1];
    if (j > 0) div -= (double)dy[idx] - (double)dy[idx - nx];
    if (k > 0) div -= (double)dz[idx] - (double)dz[idx - (long long)nx * ny];
    const double r = div - 4.0 * M_PI * rho[idx];
    if (res) res[idx] = r;
    if (i >= lo && j >= lo && k >= lo && i <= nx - 1 - lo && j <= ny - 1 - lo && k <= nz - 1 - lo) worst = fabs(r);
  }
  // warp maximum, one atomic per warp
  for (int off = 16; off > 0; off >>= 1) worst = fmax(worst, __shfl_down_sync(0xffffffffu, worst, off));
  if ((threadIdx.x & 31) == 0 && worst > 0.0) atomicMax(maxabs, (unsigned long long)__double_as_longlong(worst));
}

// Sums and maxima of the invariant statistics (maxima of non-negative doubles as bit patterns).
struct InvAcc {
  unsigned long long n, tracked;
  double norm_sum, e_sum, l_sum;
  unsigned long long norm_max, e_max, l_max;
  unsigned long long max_id;
};

__device__ __forceinline__ void warp_sum_max(double v, double* sum, unsigned long long* mx) {
  double s = v, m = v;
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, off);
    m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  }
  if ((threadIdx.x & 31) == 0) {
    if (s != 0.0) atomicAdd(sum, s);
    if (m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
  }
}

template <typename T>
__global__ void k_max_id(const Particles<T> P, unsigned long long* max_id) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = i < P.n && i < (long long)(*P.n_dev) && P.key[i] != kDead;
  // ids are 32-bit: one warp maximum, then one atomic per warp (a live id may be 0, so the warp
  // publishes only when it has a live particle)
  const unsigned v = live ? P.id[i] : 0u;
  const unsigned m = __reduce_max_sync(0xffffffffu, v);
  const unsigned any = __ballot_sync(0xffffffffu, live);
  if (any && (threadIdx.x & 31) == 0) atomicMax(max_id, (unsigned long long)m);
}

// mode 0: record E and L of the tracked particles (id % stride == 0) at slot id / stride; mode 1:
// compare with the recorded values.  The norm statistics cover every live particle.
template <typename T>
__global__ void k_invariants(const Grid g, const Particles<T> P, int mode, int stride, double* __restrict__ e0,
                             double* __restrict__ l0, long long nslots, InvAcc* acc) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = i < P.n && i < (long long)(*P.n_dev) && P.key[i] != kDead;
  double norm = 0.0, de = 0.0, dl = 0.0;
  bool cmp = false;
  if (live) {
    const double X = (double)P.x[0][i] - g.xc, Y = (double)P.x[1][i] - g.yc, Z = (double)P.x[2][i] - g.zc;
    const double u[4] = {(double)P.u[0][i], (double)P.u[1][i], (double)P.u[2][i], (double)P.u[3][i]};
    const Kerr<double> K = kerr_eval<double>(X, Y, Z, g.m, g.a);
    const double f = K.flat ? 0.0 : K.f;
    // u_m = g_mn u^n = eta_mn u^n + f k_m (k.u), k_4 = 1
    const double s = K.k0 * u[0] + K.k1 * u[1] + K.k2 * u[2] + u[3];
    const double uc[4] = {u[0] + f * s * K.k0, u[1] + f * s * K.k1, u[2] + f * s * K.k2, -u[3] + f * s};
    const double c2 = g.c * g.c;
    norm = fabs(u[0] * uc[0] + u[1] * uc[1] + u[2] * uc[2] + u[3] * uc[3] + c2) / c2;
    const double E = -uc[3], L = X * uc[1] - Y * uc[0];
    const unsigned id = P.id[i];
    if (id % (unsigned)stride == 0u) {
      const long long slot = id / (unsigned)stride;
      if (slot < nslots) {
        if (mode == 0) {
          e0[slot] = E;
          l0[slot] = L;
        } else if (!isnan(e0[slot])) {
          cmp = true;
          de = fabs(E - e0[slot]) / g.c;
          dl = fabs(L - l0[slot]) / g.c;
        }
      }
    }
  }
  const unsigned nl = __popc(__ballot_sync(0xffffffffu, live)), nc = __popc(__ballot_sync(0xffffffffu, cmp));
  if ((threadIdx.x & 31) == 0) {
    if (nl) atomicAdd(&acc->n, (unsigned long long)nl);
    if (nc) atomicAdd(&acc->tracked, (unsigned long long)nc);
  }
  warp_sum_max(norm, &acc->norm_sum, &acc->norm_max);
  warp_sum_max(de, &acc->e_sum, &acc->e_max);
  warp_sum_max(dl, &acc->l_sum, &acc->l_max);
}

}  // namespace

template <typename T>
void launch_invariants(const Grid& g, const Particles<T>& P, int mode, int stride, double* e0, double* l0,
                       long long nslots, void* acc, cudaStream_t stream) {
  if (P.n <= 0) return;
  k_invariants<T><<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(g, P, mode, stride, e0, l0, nslots,
                                                                     static_cast<InvAcc*>(acc));
}

template <typename T>
void launch_max_id(const Particles<T>& P, unsigned long long* max_id, cudaStream_t stream) {
  if (P.n <= 0) return;
  k_max_id<T><<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(P, max_id);
}

size_t invariant_acc_bytes() { return sizeof(InvAcc); }

template void launch_invariants<float>(const Grid&, const Particles<float>&, int, int, double*, double*, long long,
                                       void*, cudaStream_t);
template void launch_invariants<double>(const Grid&, const Particles<double>&, int, int, double*, double*,
                                        long long, void*, cudaStream_t);
template void launch_max_id<float>(const Particles<float>&, unsigned long long*, cudaStream_t);
template void launch_max_id<double>(const Particles<double>&, unsigned long long*, cudaStream_t);

template <typename T>
void launch_charge_density(const Particles<T>& P, double q, const Grid& g, bool with_gamma, double* rho,
                           cudaStream_t stream) {
  if (P.n <= 0) return;
  k_charge_density<T><<<(unsigned)((P.n + 255) / 256), 256, 0, stream>>>(P, q, g.nx, g.ny, g.nz, 1.0 / g.c,
                                                                         with_gamma, rho);
}

template <typename T>
void launch_gauss(const Fields<T>& F, const double* rho, const Grid& g, int lo, double* res,
                  unsigned long long* maxabs, cudaStream_t stream) {
  k_gauss<T><<<(unsigned)((g.ncell + 255) / 256), 256, 0, stream>>>(F.d[0], F.d[1], F.d[2], rho, g.nx, g.ny, g.nz,
                                                                     lo, res, maxabs);
}

template void launch_charge_density<float>(const Particles<float>&, double, const Grid&, bool, double*,
                                           cudaStream_t);
template void launch_charge_density<double>(const Particles<double>&, double, const Grid&, bool, double*,
                                            cudaStream_t);
template void launch_gauss<float>(const Fields<float>&, const double*, const Grid&, int, double*,
                                  unsigned long long*, cudaStream_t);
template void launch_gauss<double>(const Fields<double>&, const double*, const Grid&, int, double*,
                                   unsigned long long*, cudaStream_t);

}  // namespace grpic
