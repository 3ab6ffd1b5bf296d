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
#include <cmath>

#include "common.cuh"

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

}  // namespace

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
