// Per-cell polynomial fits of the face-area integrand of Eq. 18 for the far-field deposit.
//
// The integrand sqrt(g_II g_JJ - g_IJ^2) = sqrt(1 + f (1 - k_K^2)) of the face normal to axis K
// depends on position only (the metric is stationary), so each cell can carry, per K, a
// polynomial in the cell fractions (u, v, w) along (I, J, K) = (K+1, K+2, K) mod 3:
//     g_K(u, v, w) ~ sum_{i+j+k <= 4} c_ijk u^i v^j w^k.
// A face plane w of that cell, split at (u, v), then has its four sub-rectangle AREAs in closed
// form (the mean of t^i over [0, u] is u^i / (i+1), over [u, 1] it is (1 + u + ... + u^i) / (i+1)),
// with no evaluation of the metric per particle.
//
// The fit: the integrand at the 5 x 5 x 5 Chebyshev points of the cell, the tensor Chebyshev
// interpolant, its terms of total degree <= 4, re-expanded in monomials of (u, v, w).  Far from the
// hole (particles at R >= table_radius) the truncated terms, which scale as m / r^6, move the
// weights W of Eq. 18 by a few 1e-9 from Gauss-Legendre quadrature at Q = 2 on every sub-rectangle.
// The samples and the fit are FP32, like the per-node integrand of the FP32 deposit: the fit is
// of delta = g - 1, formed as x / (1 + sqrt(1 + x)) with x = f (1 - k_K^2), which keeps its
// relative precision, and the 1 goes back into the constant term.  Near the hole the push keeps
// the per-node quadrature.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace grpic {

namespace {

constexpr int kN = 5;  // Chebyshev points per axis (degree 4)

// t_i: the Chebyshev points of the first kind on [0, 1]; cheb[p][i]: value i -> coefficient p of
// T_p(2t - 1) (discrete orthogonality); mono[a][p]: coefficient of t^a in T_p(2t - 1).  Formed in
// FP64 on the host, passed in FP32.
struct FitMatrices {
  float t[kN];
  float cheb[kN][kN];
  float mono[kN][kN];
};

FitMatrices fit_matrices() {
  FitMatrices M{};
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < kN; ++i) {
    const double t = 0.5 - 0.5 * std::cos((2 * i + 1) * pi / (2 * kN));
    M.t[i] = (float)t;
    // c_p = (2 - [p = 0]) / N sum_i f_i T_p(s_i) at the points s_i = 2 t_i - 1 = -cos((2i+1) pi / 2N)
    const double s = 2.0 * t - 1.0;
    double tp = 1.0, tq = s;  // T_p(s), T_{p+1}(s)
    for (int p = 0; p < kN; ++p) {
      M.cheb[p][i] = (float)((p == 0 ? 1.0 : 2.0) / kN * tp);
      const double tn = 2.0 * s * tq - tp;
      tp = tq;
      tq = tn;
    }
  }
  // T_0 = 1, T_1 = s, T_{p+1} = 2 s T_p - T_{p-1} with s = 2t - 1, as polynomials in t
  double T[kN][kN] = {};
  T[0][0] = 1.0;
  T[1][0] = -1.0;
  T[1][1] = 2.0;
  for (int p = 1; p + 1 < kN; ++p)
    for (int a = 0; a < kN; ++a) {
      const double sT = (a > 0 ? 2.0 * T[p][a - 1] : 0.0) - T[p][a];  // (2t - 1) T_p, coefficient of t^a
      T[p + 1][a] = 2.0 * sT - T[p - 1][a];
    }
  for (int a = 0; a < kN; ++a)
    for (int p = 0; p < kN; ++p) M.mono[a][p] = (float)T[p][a];
  return M;
}

// delta_K = sqrt(1 + f (1 - k_K^2)) - 1, the Eq. 18 integrand minus one, of the three face
// orientations at (X, Y, Z) (offsets from the centre).  r^2 from Eq. 6 in its cancellation-free
// form, f = 2 m r / D at the root (Sigma = r^2 D); r = 0 (the disk z = 0, R <= a) takes the flat
// limit.
__device__ __forceinline__ void deltas(float X, float Y, float Z, float m, float a, float out[3]) {
  const float a2 = a * a, q = a2 * Z * Z;
  const float p = fmaf(X, X, fmaf(Y, Y, fmaf(Z, Z, -a2)));
  const float D = sqrtf(fmaf(p, p, 4.f * q));
  const float r2 = p >= 0.f ? 0.5f * (p + D) : 2.f * q / (D - p);
  if (!(r2 > 0.f) || !(D > 0.f)) {
    out[0] = out[1] = out[2] = 0.f;
    return;
  }
  const float r = sqrtf(r2);
  const float f = 2.f * m * r / D;
  const float rho2 = r2 + a2;
  const float kx = (r * X - a * Y) / rho2, ky = (r * Y + a * X) / rho2;
  const float x[3] = {f * (1.f - kx * kx), f * (1.f - ky * ky), f * (r2 - Z * Z) / r2};
#pragma unroll
  for (int K = 0; K < 3; ++K) out[K] = x[K] / (1.f + sqrtf(1.f + x[K]));
}

// One thread per cell: the fits of its three face orientations, kAreaTableStride float4 per cell
// (layout in common.cuh).  Cells past n-2 on an axis (never a deposit cell) are zeroed.
__global__ void k_area_table(const Grid g, const FitMatrices M, float4* __restrict__ tab) {
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= g.ncell) return;
  const int cx = (int)(cell % g.nx), cy = (int)((cell / g.nx) % g.ny);
  const int cz = (int)(cell / ((long long)g.nx * g.ny));
  float* out = reinterpret_cast<float*>(tab + cell * kAreaTableStride);
  if (cx > g.nx - 2 || cy > g.ny - 2 || cz > g.nz - 2) {
    for (int q = 0; q < 4 * kAreaTableStride; ++q) out[q] = 0.f;
    return;
  }
  // offsets of the cell's corner from the centre (exact in FP64, then rounded once)
  const float ox = (float)(cx - g.xc), oy = (float)(cy - g.yc), oz = (float)(cz - g.zc);
  const float m = (float)g.m, a = (float)g.a;
  float val[3][kN][kN][kN];  // [K][ix][iy][iz]
  for (int ix = 0; ix < kN; ++ix)
    for (int iy = 0; iy < kN; ++iy)
      for (int iz = 0; iz < kN; ++iz) {
        float o[3];
        deltas(ox + M.t[ix], oy + M.t[iy], oz + M.t[iz], m, a, o);
        val[0][ix][iy][iz] = o[0];
        val[1][ix][iy][iz] = o[1];
        val[2][ix][iy][iz] = o[2];
      }
  for (int K = 0; K < 3; ++K) {
    // A[iu][iv][s]: Chebyshev coefficients along w; then along v, then along u (total degree <= 4)
    float A[kN][kN][kN], C[kN][kN][kN];
    for (int iu = 0; iu < kN; ++iu)
      for (int iv = 0; iv < kN; ++iv)
        for (int s = 0; s < kN; ++s) {
          float acc = 0.f;
          for (int iw = 0; iw < kN; ++iw) {
            int p3[3];
            p3[K] = iw;
            p3[(K + 1) % 3] = iu;
            p3[(K + 2) % 3] = iv;
            acc = fmaf(M.cheb[s][iw], val[K][p3[0]][p3[1]][p3[2]], acc);
          }
          A[iu][iv][s] = acc;
        }
    for (int iu = 0; iu < kN; ++iu)
      for (int q = 0; q < kN; ++q)
        for (int s = 0; s < kN; ++s) {
          float acc = 0.f;
          if (q + s < kN)
            for (int iv = 0; iv < kN; ++iv) acc = fmaf(M.cheb[q][iv], A[iu][iv][s], acc);
          C[iu][q][s] = acc;
        }
    for (int p = 0; p < kN; ++p)
      for (int q = 0; q < kN; ++q)
        for (int s = 0; s < kN; ++s) {
          float acc = 0.f;
          if (p + q + s < kN)
            for (int iu = 0; iu < kN; ++iu) acc = fmaf(M.cheb[p][iu], C[iu][q][s], acc);
          A[p][q][s] = acc;  // Chebyshev coefficients of total degree <= 4, zero above
        }
    // re-expansion in monomials, one axis at a time (T_p(2t - 1) has degree p, so the total
    // degree stays <= 4)
    for (int a_ = 0; a_ < kN; ++a_)
      for (int q = 0; q < kN; ++q)
        for (int s = 0; s < kN; ++s) {
          float acc = 0.f;
          for (int p = a_; p < kN; ++p) acc = fmaf(M.mono[a_][p], A[p][q][s], acc);
          C[a_][q][s] = acc;
        }
    for (int a_ = 0; a_ < kN; ++a_)
      for (int b = 0; b < kN; ++b)
        for (int s = 0; s < kN; ++s) {
          float acc = 0.f;
          for (int q = b; q < kN; ++q) acc = fmaf(M.mono[b][q], C[a_][q][s], acc);
          A[a_][b][s] = acc;
        }
    float cf[kFitTerms];
    int n = 0;
    for (int j = 0; j < kN; ++j)
      for (int i = 0; i + j < kN; ++i)
        for (int k = 0; i + j + k < kN; ++k) {
          float acc = 0.f;
          for (int s = k; s < kN; ++s) acc = fmaf(M.mono[k][s], A[i][j][s], acc);
          cf[n++] = (i + j + k == 0) ? 1.f + acc : acc;  // the integrand is 1 + delta
        }
    float* o = out + 20 * K;
    o[0] = cf[0];
    o[1] = cf[1];
    o[2] = cf[5];
    o[3] = cf[15];
    __half* h = reinterpret_cast<__half*>(o + 4);
    int q = 0;
    for (int t = 0; t < kFitTerms; ++t)
      if (!fit_term_fp32(t)) h[q++] = __float2half_rn(cf[t]);
    h[q] = __float2half_rn(0.f);
  }
  for (int q = 60; q < 64; ++q) out[q] = 0.f;
}

}  // namespace

double table_radius(const Grid& g) {
  const double rn = near_radius(g);
  return g.m > 0.0 ? std::max(rn, 4.0 + std::pow(g.m / 4.5e-7, 1.0 / 6.0)) : rn;
}

void launch_area_table(const Grid& g, float4* tab, cudaStream_t st) {
  const FitMatrices M = fit_matrices();
  const unsigned nb = (unsigned)((g.ncell + 127) / 128);
  k_area_table<<<nb, 128, 0, st>>>(g, M, tab);
}

}  // namespace grpic
