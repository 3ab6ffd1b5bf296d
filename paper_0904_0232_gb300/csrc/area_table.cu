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
// The fit: the integrand in FP64 at the 5 x 5 x 5 Chebyshev points of the cell, the tensor
// Chebyshev interpolant, its terms of total degree <= 4, re-expanded in monomials of (u, v, w).
// Far from the hole (particles at R >= table_radius) the weights W of Eq. 18 it gives agree with
// Gauss-Legendre quadrature at Q = 2 on every sub-rectangle to a few 1e-9: the truncated terms
// scale as m / r^6.  Near the hole the push keeps the per-node quadrature.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "metric.cuh"

namespace grpic {

namespace {

constexpr int kN = 5;  // Chebyshev points per axis (degree 4)

// t_i: the Chebyshev points of the first kind on [0, 1]; cheb[p][i]: value i -> coefficient p of
// T_p(2t - 1) (discrete orthogonality); mono[a][p]: coefficient of t^a in T_p(2t - 1).
struct FitMatrices {
  double t[kN];
  double cheb[kN][kN];
  double mono[kN][kN];
};

FitMatrices fit_matrices() {
  FitMatrices M{};
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < kN; ++i) {
    M.t[i] = 0.5 - 0.5 * std::cos((2 * i + 1) * pi / (2 * kN));
    // c_p = (2 - [p = 0]) / N sum_i f_i T_p(s_i) at the points s_i = 2 t_i - 1 = -cos((2i+1) pi / 2N)
    const double s = 2.0 * M.t[i] - 1.0;
    double tp = 1.0, tq = s;  // T_p(s), T_{p+1}(s)
    for (int p = 0; p < kN; ++p) {
      M.cheb[p][i] = (p == 0 ? 1.0 : 2.0) / kN * tp;
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
    for (int p = 0; p < kN; ++p) M.mono[a][p] = T[p][a];
  return M;
}

// Eq. 18 integrand of the three face orientations at (X, Y, Z) (offsets from the centre), FP64
// with the seeded reciprocal and root (a Newton step from the FP32 value: ~1e-14 relative).
__device__ __forceinline__ void integrands(double X, double Y, double Z, double m, double a, double out[3]) {
  double D;
  const double r2 = kerr_r2<double, SeededOps64>(X, Y, Z, a, &D);
  if (!(r2 > 0.0)) {
    out[0] = out[1] = out[2] = 1.0;
    return;
  }
  const double a2 = a * a;
  const double r = SeededOps64::root(r2);
  const double inv_sig = SeededOps64::rcp(r2 * r2 + a2 * Z * Z);
  const double irho2 = SeededOps64::rcp(r2 + a2);
  const double tm = 2.0 * m * r;
  const double kx = (r * X - a * Y) * irho2, ky = (r * Y + a * X) * irho2;
  out[0] = SeededOps64::root(1.0 + tm * r2 * (1.0 - kx * kx) * inv_sig);
  out[1] = SeededOps64::root(1.0 + tm * r2 * (1.0 - ky * ky) * inv_sig);
  out[2] = SeededOps64::root(1.0 + tm * (r2 - Z * Z) * inv_sig);
}

// One thread per cell: the fits of its three face orientations, kAreaTableStride float4 per cell
// (36 floats per K: for j = 0..4, i = 0..4-j, the coefficients of w^0..w^(4-i-j) of u^i v^j; the
// 36th is zero).  Cells past n-2 on an axis (never a deposit cell) are zeroed.
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
  double val[3][kN][kN][kN];  // [K][ix][iy][iz]
  for (int ix = 0; ix < kN; ++ix)
    for (int iy = 0; iy < kN; ++iy)
      for (int iz = 0; iz < kN; ++iz) {
        double o[3];
        integrands(cx + M.t[ix] - g.xc, cy + M.t[iy] - g.yc, cz + M.t[iz] - g.zc, g.m, g.a, o);
        val[0][ix][iy][iz] = o[0];
        val[1][ix][iy][iz] = o[1];
        val[2][ix][iy][iz] = o[2];
      }
  for (int K = 0; K < 3; ++K) {
    // A[iu][iv][s]: Chebyshev coefficients along w; then along v, then along u (total degree <= 4)
    double A[kN][kN][kN], C[kN][kN][kN];
    for (int iu = 0; iu < kN; ++iu)
      for (int iv = 0; iv < kN; ++iv)
        for (int s = 0; s < kN; ++s) {
          double acc = 0.0;
          for (int iw = 0; iw < kN; ++iw) {
            int p3[3];
            p3[K] = iw;
            p3[(K + 1) % 3] = iu;
            p3[(K + 2) % 3] = iv;
            acc += M.cheb[s][iw] * val[K][p3[0]][p3[1]][p3[2]];
          }
          A[iu][iv][s] = acc;
        }
    for (int iu = 0; iu < kN; ++iu)
      for (int q = 0; q < kN; ++q)
        for (int s = 0; s < kN; ++s) {
          double acc = 0.0;
          if (q + s < kN)
            for (int iv = 0; iv < kN; ++iv) acc += M.cheb[q][iv] * A[iu][iv][s];
          C[iu][q][s] = acc;
        }
    for (int p = 0; p < kN; ++p)
      for (int q = 0; q < kN; ++q)
        for (int s = 0; s < kN; ++s) {
          double acc = 0.0;
          if (p + q + s < kN)
            for (int iu = 0; iu < kN; ++iu) acc += M.cheb[p][iu] * C[iu][q][s];
          A[p][q][s] = acc;  // Chebyshev coefficients of total degree <= 4, zero above
        }
    // re-expansion in monomials, one axis at a time (T_p(2t - 1) has degree p, so the total
    // degree stays <= 4)
    for (int a = 0; a < kN; ++a)
      for (int q = 0; q < kN; ++q)
        for (int s = 0; s < kN; ++s) {
          double acc = 0.0;
          for (int p = a; p < kN; ++p) acc += M.mono[a][p] * A[p][q][s];
          C[a][q][s] = acc;
        }
    for (int a = 0; a < kN; ++a)
      for (int b = 0; b < kN; ++b)
        for (int s = 0; s < kN; ++s) {
          double acc = 0.0;
          for (int q = b; q < kN; ++q) acc += M.mono[b][q] * C[a][q][s];
          A[a][b][s] = acc;
        }
    float* o = out + 36 * K;
    int n = 0;
    for (int j = 0; j < kN; ++j)
      for (int i = 0; i + j < kN; ++i)
        for (int k = 0; i + j + k < kN; ++k) {
          double acc = 0.0;
          for (int s = k; s < kN; ++s) acc += M.mono[k][s] * A[i][j][s];
          o[n++] = (float)acc;
        }
    o[35] = 0.f;
  }
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
