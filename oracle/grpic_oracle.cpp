/*
 * GRPIC oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of one timestep of the general-relativistic
 * electromagnetic particle-in-cell method of Watson & Nishikawa, "A Method for
 * Incorporating General Relativity in Electromagnetic Particle-in-Cell Code"
 * (arXiv:0904.0232).  Only the test suite, the smoke check and the benchmark's CPU
 * baseline / reference arm may load it.  It shares no code, header, table or helper
 * with the CUDA library: every formula here is written from the paper directly.
 *
 * Deliberate differences from how a fast implementation would compute the same things
 * (so that the two can check each other):
 *   - Christoffel symbols are formed as all 64 Gamma^a_{mn} = 1/2 g^{ab}(d_m g_bn + d_n g_bm
 *     - d_b g_mn), with d g obtained by forward-mode dual numbers through the metric of
 *     Eqs. 4-6, and g^{ab} by numerical Gauss-Jordan inversion.
 *   - The missing components of the field tensor at a point are found by solving the
 *     index-lowering relation F_{mn} = g_{ma} g_{nb} F^{ab} numerically (3x3 linear solve).
 *   - The face-area integrand of Eq. 18 is sqrt(g_II g_JJ - g_IJ^2) read off the full
 *     4x4 metric.
 *
 * Readings of passages the paper leaves open (numbering as in the design notes):
 *   A1  RK4 (Sec. 3.3, steps 1-4): classical RK4 in proper time with one step
 *       h = dt / gamma_1 per particle-step, gamma_1 from Eq. 16 at (x_n, u_n).
 *   A2  Eq. 16 with a negative square-root argument (or gamma <= 0) falls back to
 *       gamma_1 = u^4/c and the event is counted.
 *   A3  Eq. 5 with dt -> dx^4 = c dt; the paper's sign of the spin term is kept.
 *   A5  Sub-volumes of Sec. 3.3 use sqrt(-det g) of the 4-metric.  For Eq. 4, det g = -1
 *       identically, so the CIC weights are exactly trilinear; orc_volume_weights()
 *       integrates sqrt(-det g) numerically so a test can check that identity.
 *   A6  The Christoffel terms of Eq. 11 are evaluated as Gamma^a_{cb} F^{cb} +
 *       Gamma^b_{bc} F^{ac} (index-garble reading); both vanish identically here.
 *   A7  Prognostic fields: covariant F_{yz}, F_{zx}, F_{xy} on faces (Eq. 10 advances
 *       them), contravariant F^{x4}, F^{y4}, F^{z4} on edges (Eq. 12 advances them).  At
 *       any lattice point the other components are the mean of the nearest 2, 4 or 8
 *       points of their own lattice.
 *   A8  Eq. 12 takes the sign of the continuous Eq. 11: F^{a4} += (4 pi/c J^a - ...) dx^4.
 *   A9  The divergence in Eq. 11 sums over spatial nu only.
 *   A10 The Lorentz term is (q/m) F^a_b u^b literally.
 *   A11 Each prognostic component is interpolated from its own staggered lattice, then
 *       converted and index-shifted with g at the particle.
 *   A12 Face weights of Sec. 4: the I-J plane sits at the segment midpoint's K
 *       coordinate; FACE_AREA is the sum of the four sub-areas; Q x Q Gauss-Legendre.
 *   A13 J = rho u = rho gamma v: the Umeda flux is multiplied by gamma_bar =
 *       (u^4_n + u^4_{n+1}) / (2c) unless ORC_NO_GAMMA_IN_J is set.
 *   A15 Particles are removed when r <= r_+ or a coordinate leaves [1, N-2].  Field
 *       components on the outer two index layers, or at points with r < r_excise (default
 *       r_+: the whole inside of the horizon), are not advanced; field conversions at points
 *       with r < r_excise use the flat metric.
 *       A metric evaluated where r = 0 exactly (the disk z = 0, R <= a) is flat.
 *   A16 Particles are pushed with the fields present after the first B half-step;
 *       J is deposited from x_n -> x_{n+1}.
 *   A21 Time levels of the field tensor in Eqs. 9-12 (unstated): time-centred.  The stored b
 *       lags d by half a step.  First half-step: b^n = b^{n-1/2} - (dx^4/2) curl e(b^{n-1/2}, d^n);
 *       second: b^{n+1/2} = b^{n-1/2} - dx^4 curl e(b^n, d^n); E step: the contravariant tensor
 *       in the divergence is taken at (b^{n+1/2}, d*) with the midpoint predictor
 *       d* = d^n + (dx^4/2) rhs(b^{n+1/2}, d^n).  In Kerr-Schild coordinates e depends on b and
 *       h on d (the shift terms), and evaluating them at each half-step's own start value
 *       (ORC_LITERAL_HALF_STEPS) is a forward-Euler step of a centred advection term, which grows
 *       without bound near the horizon.
 *   A23 Absorbing layers (optional; off unless absorb_inner or absorb_outer > 0; the paper states
 *       no boundary condition).  After the second B half-step and the E step every advanced
 *       point takes F0 + (1 - kappa)(F - F0), F0 the field as last set, kappa the larger of an
 *       inner layer's absorb_inner (r_+ - r)/(r_+ - r_excise) for r_excise <= r < r_+ (r_excise
 *       defaulting to r_+/2 then) and an outer layer's absorb_outer ((W + 1 - s)/W)^2 over the
 *       W cells next to the frozen faces (s = 1 at the first advanced cell).  Held fields reflect;
 *       with a rapidly rotating hole, reflection inside the horizon feeds a mode growing next to
 *       it, and frozen faces where the metric is far from flat feed one at the box edges.
 *
 *   A24 (not in the paper) A grid may be one slab of a larger run: planes z_origin ..
 *       z_origin + nz - 1 of nz_total, the hole at the whole run's centre.  Everything else is as
 *       for a whole grid; a driver that splits a run refreshes the slabs' overlapping planes.
 *
 * Parity status: every function is pinned by a CPU test against closed forms, invariants
 * or brute force.  The RK4 steps exactly as printed in Sec. 3.3 have no consistent reading
 * (parity unpinned for that literal form).  For an ablation ORC_RK4_AS_PRINTED takes the
 * printed steps with only the missing x_n and u_n added to the final sums (stage proper-time
 * steps dt/(2 gamma_1), dt/gamma_2, dt/gamma_3, dt/(2 gamma_4); trapezoid stage velocities);
 * its stage weights add up to 5/6 of a step, which the tests show.
 *
 * Array layout at this boundary: a grid array is nz*ny*nx doubles, index (k*ny + j)*nx + i.
 * Particle arrays are planar: x4 holds x^1[0..n), x^2[0..n), x^3[0..n), x^4[0..n); u4 alike.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846;

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID = 1,
  ORC_ERR_CFL = 4,
  ORC_ERR_NONFINITE = 5,
};

enum {
  ORC_NO_GAMMA_IN_J = 1u,   // A13 off: plain Umeda flux (charge conserving in flat space)
  ORC_NO_GAMMA_TERMS = 2u,  // skip the (identically zero) Christoffel terms of Eq. 11
  ORC_FROZEN_FIELDS = 4u,   // test-particle runs: the cycle does not advance the fields
  ORC_LITERAL_HALF_STEPS = 8u,  // each B half-step and the E step explicit in their own start values
  ORC_RK4_AS_PRINTED = 16u,     // ablation: the printed RK4 steps, finals with x_n, u_n added
  ORC_ANALYTIC_WALD = 32u,      // test-particle pins: the Lorentz term takes Wald's field at the particle
};

// ---------------------------------------------------------------------------------------
// Forward-mode dual numbers carrying d/dx, d/dy, d/dz.  The metric does not depend on x^4,
// so its x^4 derivative is zero and is not carried.
// ---------------------------------------------------------------------------------------
struct Dual {
  double v;
  double d[3];
  Dual() : v(0.0), d{0.0, 0.0, 0.0} {}
  Dual(double c) : v(c), d{0.0, 0.0, 0.0} {}  // NOLINT: implicit on purpose
};
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v + b.v;
  for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v - b.v;
  for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
inline Dual operator-(const Dual& a) {
  Dual r;
  r.v = -a.v;
  for (int i = 0; i < 3; ++i) r.d[i] = -a.d[i];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v * b.v;
  for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v / b.v;
  for (int i = 0; i < 3; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
inline Dual sqrt(const Dual& a) {
  Dual r;
  r.v = std::sqrt(a.v);
  const double h = r.v > 0.0 ? 0.5 / r.v : 0.0;
  for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] * h;
  return r;
}
using std::sqrt;

// ---------------------------------------------------------------------------------------
// Kerr metric in Cartesian Kerr-Schild form (Eqs. 4-6).  X is the position relative to
// the central mass; indices 0..3 = x, y, z, x^4 = c t; eta = diag(1, 1, 1, -1).
// ---------------------------------------------------------------------------------------
template <class S>
struct KerrFK {
  S r, f;
  S k[4];
  bool flat;
};

template <class S>
KerrFK<S> kerr_fk(const S X[3], double m, double a) {
  const S& x = X[0];
  const S& y = X[1];
  const S& z = X[2];
  KerrFK<S> o;
  // Eq. 6: r^4 - (R^2 - a^2) r^2 - a^2 z^2 = 0, a quadratic in r^2; its non-negative root.
  S R2 = x * x + y * y + z * z;
  S p = R2 - a * a;
  S q = a * a * z * z;
  S disc = sqrt(p * p + 4.0 * q);
  // Both branches are the same root; the second avoids cancellation when p < 0.
  S r2 = (val(p) >= 0.0) ? 0.5 * (p + disc) : (2.0 * q) / (disc - p);
  if (!(val(r2) > 0.0)) {
    o.flat = true;
    o.r = S(0.0);
    o.f = S(0.0);
    o.k[0] = S(0.0);
    o.k[1] = S(0.0);
    o.k[2] = S(0.0);
    o.k[3] = S(1.0);
    return o;
  }
  o.flat = false;
  o.r = sqrt(r2);
  // Eq. 4: coefficient 2 m r^3 / (r^4 + a^2 z^2) of k (x) k.
  o.f = 2.0 * m * o.r * r2 / (r2 * r2 + q);
  // Eq. 5 (dt -> dx^4): k = [r^2 (x dx + y dy) + a r (x dy - y dx) + (r^2 + a^2)(z dz + r dx^4)]
  //                        / ((r^2 + a^2) r)
  S den = (r2 + a * a) * o.r;
  o.k[0] = (r2 * x - a * o.r * y) / den;
  o.k[1] = (r2 * y + a * o.r * x) / den;
  o.k[2] = (r2 + a * a) * z / den;
  o.k[3] = (r2 + a * a) * o.r / den;
  return o;
}

template <class S>
void kerr_metric(const S X[3], double m, double a, S g[4][4]) {
  KerrFK<S> kf = kerr_fk(X, m, a);
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      const double eta = (mu == nu) ? (mu == 3 ? -1.0 : 1.0) : 0.0;
      g[mu][nu] = S(eta) + kf.f * kf.k[mu] * kf.k[nu];
    }
}

void flat_metric(double g[4][4]) {
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) g[mu][nu] = (mu == nu) ? (mu == 3 ? -1.0 : 1.0) : 0.0;
}

// Gauss-Jordan inversion with partial pivoting.
bool invert4(const double A[4][4], double Ai[4][4]) {
  double M[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) M[i][j] = (j < 4) ? A[i][j] : ((j - 4 == i) ? 1.0 : 0.0);
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    if (M[piv][col] == 0.0) return false;
    if (piv != col)
      for (int j = 0; j < 8; ++j) std::swap(M[piv][j], M[col][j]);
    const double inv = 1.0 / M[col][col];
    for (int j = 0; j < 8; ++j) M[col][j] *= inv;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      const double fac = M[r][col];
      for (int j = 0; j < 8; ++j) M[r][j] -= fac * M[col][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Ai[i][j] = M[i][j + 4];
  return true;
}

// Determinant by LU with partial pivoting.
double det4(const double A[4][4]) {
  double M[4][4];
  std::memcpy(M, A, sizeof(M));
  double det = 1.0;
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    if (M[piv][col] == 0.0) return 0.0;
    if (piv != col) {
      for (int j = 0; j < 4; ++j) std::swap(M[piv][j], M[col][j]);
      det = -det;
    }
    det *= M[col][col];
    for (int r = col + 1; r < 4; ++r) {
      const double fac = M[r][col] / M[col][col];
      for (int j = col; j < 4; ++j) M[r][j] -= fac * M[col][j];
    }
  }
  return det;
}

// 3x3 solve by Gaussian elimination with partial pivoting.
bool solve3(double A[3][3], double b[3], double x[3]) {
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (A[piv][col] == 0.0) return false;
    if (piv != col) {
      for (int j = 0; j < 3; ++j) std::swap(A[piv][j], A[col][j]);
      std::swap(b[piv], b[col]);
    }
    for (int r = col + 1; r < 3; ++r) {
      const double fac = A[r][col] / A[col][col];
      for (int j = col; j < 3; ++j) A[r][j] -= fac * A[col][j];
      b[r] -= fac * b[col];
    }
  }
  for (int r = 2; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < 3; ++j) s -= A[r][j] * x[j];
    x[r] = s / A[r][r];
  }
  return true;
}

void metric_at(const double X[3], double m, double a, double g[4][4]) { kerr_metric<double>(X, m, a, g); }

// d_l g_{mn} for l = 0..2 (l = 3 is zero), by dual numbers through Eqs. 4-6.
void metric_grad(const double X[3], double m, double a, double g[4][4], double dg[4][4][4]) {
  Dual Xd[3];
  for (int i = 0; i < 3; ++i) {
    Xd[i] = Dual(X[i]);
    Xd[i].d[i] = 1.0;
  }
  Dual gd[4][4];
  kerr_metric<Dual>(Xd, m, a, gd);
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      g[mu][nu] = gd[mu][nu].v;
      for (int l = 0; l < 3; ++l) dg[l][mu][nu] = gd[mu][nu].d[l];
      dg[3][mu][nu] = 0.0;
    }
}

// Christoffel symbols of the second kind, G[a][m][n] = Gamma^a_{mn} (used in Eq. 3 and Eq. 11).
void christoffel_at(const double X[3], double m, double a, double G[4][4][4]) {
  double g[4][4], dg[4][4][4], gi[4][4];
  metric_grad(X, m, a, g, dg);
  invert4(g, gi);
  for (int al = 0; al < 4; ++al)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = 0; nu < 4; ++nu) {
        double s = 0.0;
        for (int be = 0; be < 4; ++be) s += gi[al][be] * (dg[mu][be][nu] + dg[nu][be][mu] - dg[be][mu][nu]);
        G[al][mu][nu] = 0.5 * s;
      }
}

// F_{mn} = g_{ma} g_{nb} F^{ab}
void lower2(const double g[4][4], const double Fu[4][4], double Fd[4][4]) {
  double T[4][4];
  for (int mu = 0; mu < 4; ++mu)
    for (int be = 0; be < 4; ++be) {
      double s = 0.0;
      for (int al = 0; al < 4; ++al) s += g[mu][al] * Fu[al][be];
      T[mu][be] = s;
    }
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      double s = 0.0;
      for (int be = 0; be < 4; ++be) s += T[mu][be] * g[be][nu];
      Fd[mu][nu] = s;
    }
}

// Index pairs of the covariant face components: b_x = F_{yz}, b_y = F_{zx}, b_z = F_{xy}.
const int kPair[3][2] = {{1, 2}, {2, 0}, {0, 1}};

// Contravariant tensor of Eq. 8 from F^{i4} = d^i and spatial F^{yz}, F^{zx}, F^{xy} = h.
void build_up(const double h[3], const double d[3], double Fu[4][4]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Fu[i][j] = 0.0;
  for (int i = 0; i < 3; ++i) {
    Fu[i][3] = d[i];
    Fu[3][i] = -d[i];
  }
  for (int q = 0; q < 3; ++q) {
    Fu[kPair[q][0]][kPair[q][1]] = h[q];
    Fu[kPair[q][1]][kPair[q][0]] = -h[q];
  }
}

// Given g, covariant spatial F_{yz}, F_{zx}, F_{xy} (b) and contravariant F^{x4}, F^{y4},
// F^{z4} (d) at one point, find the full tensor: solve the (linear) lowering relation for
// the contravariant spatial components, then lower the whole tensor.
bool complete_tensor(const double g[4][4], const double b[3], const double d[3], double Fu[4][4], double Fd[4][4]) {
  const double zero[3] = {0.0, 0.0, 0.0};
  double F0u[4][4], F0d[4][4];
  build_up(zero, d, F0u);
  lower2(g, F0u, F0d);
  double L[3][3], rhs[3];
  for (int q = 0; q < 3; ++q) {
    double e[3] = {0.0, 0.0, 0.0};
    e[q] = 1.0;
    double Tu[4][4], Td[4][4];
    build_up(e, d, Tu);
    lower2(g, Tu, Td);
    for (int p = 0; p < 3; ++p) L[p][q] = Td[kPair[p][0]][kPair[p][1]] - F0d[kPair[p][0]][kPair[p][1]];
  }
  for (int p = 0; p < 3; ++p) rhs[p] = b[p] - F0d[kPair[p][0]][kPair[p][1]];
  double h[3];
  if (!solve3(L, rhs, h)) return false;
  build_up(h, d, Fu);
  lower2(g, Fu, Fd);
  return true;
}

// Eq. 16: gamma_i = [u^4/c + sqrt((u^4/c)^2 + 4 a^4 dt/(2c))] / 2, with reading A2.
double gamma_f(double u4, double a4, double c, double dt, int* fallback) {
  const double w = u4 / c;
  const double arg = w * w + 4.0 * a4 * (dt / (2.0 * c));
  double gam = -1.0;
  if (arg >= 0.0) gam = 0.5 * (w + std::sqrt(arg));
  if (!(gam > 0.0) || !std::isfinite(gam)) {
    if (fallback) *fallback = 1;
    return w;
  }
  if (fallback) *fallback = 0;
  return gam;
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on the Legendre polynomial
// P_Q (three-term recurrence), weight 2 / ((1 - z^2) P_Q'(z)^2).
void legendre_pair(int Q, double z, double* pq, double* dpq) {
  double p1 = 1.0, p2 = 0.0;
  for (int j = 1; j <= Q; ++j) {
    const double p3 = p2;
    p2 = p1;
    p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
  }
  *pq = p1;                                  // P_Q(z)
  *dpq = Q * (z * p1 - p2) / (z * z - 1.0);  // P_Q'(z)
}

void gauss_legendre(int Q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(Q, 0.0);
  w.assign(Q, 0.0);
  for (int i = 0; i < Q; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (Q + 0.5));
    double pq = 0.0, dpq = 1.0;
    for (int it = 0; it < 100; ++it) {
      legendre_pair(Q, z, &pq, &dpq);
      const double dz = pq / dpq;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_pair(Q, z, &pq, &dpq);
    x[Q - 1 - i] = z;  // cos() seeds run from +1 down to -1
    w[Q - 1 - i] = 2.0 / ((1.0 - z * z) * dpq * dpq);
  }
}

// Lattice offsets, in half cells, of the six prognostic components.
// 0,1,2 = F^{x4}, F^{y4}, F^{z4} (contravariant, on edges); 3,4,5 = F_{yz}, F_{zx}, F_{xy}
// (covariant, on faces).
const int kHalf[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

struct Species {
  double qm = 0.0, qmacro = 0.0;
  std::vector<double> x[4], u[4];
  std::vector<uint32_t> id;
  // start and end positions of every particle of the last push (removed ones included)
  std::vector<double> last_x0[3], last_x1[3];
  std::vector<uint32_t> last_id;
};

}  // namespace

extern "C" {

typedef struct {
  int nx, ny, nz;
  double m, a, c, dt;
  int quad_order;
  double r_excise;  // <= 0: r_+ (r_+/2 with an inner absorbing layer)
  unsigned flags;
  int threads;  // <= 0: all available
  double absorb_inner, absorb_outer;  // A23: relaxation per step at the layers' deepest points (0: none)
  int absorb_width;                   // outer layer width in cells (<= 0: 8)
  // A24: this grid as planes z_origin .. z_origin + nz - 1 of a run whose grid has nz_total planes
  // (0: nz); the hole sits at the centre of the whole run's grid
  int z_origin, nz_total;
} orc_config;

}  // extern "C"

namespace {

void wald_field(const double X[3], double m, double a, double B0, double Fd[4][4], double Fu[4][4]);

struct Ctx {
  orc_config cfg{};
  double Xc[3]{};
  double r_plus = 0.0, r_exc = 0.0;
  int n[3]{};
  size_t ncell = 0;
  std::vector<double> F[6];
  std::vector<double> Fprev[3];  // b^{n-1/2} kept by the first B half-step (A21)
  std::vector<double> F0[6];     // target of the absorbing layers (A23), kept only with layers
  double r_abs = 0.0;            // outer radius of the inner absorbing layer (r_+)
  int w_out = 8;                 // outer absorbing layer width
  std::vector<double> J[3];
  std::vector<Species> sp;
  std::vector<double> glx, glw;
  long long stat_removed_horizon = 0, stat_removed_outer = 0, stat_fallback = 0, stat_steps = 0;
  double gterm_max = 0.0, gterm_scale = 0.0;
  double wald_B0 = 0.0;  // field strength of ORC_ANALYTIC_WALD

  size_t idx(int i, int j, int k) const { return ((size_t)k * n[1] + j) * n[0] + i; }

  int nthreads() const {
    int t = cfg.threads;
#ifdef _OPENMP
    if (t <= 0) t = omp_get_max_threads();
#else
    t = 1;
#endif
    return t < 1 ? 1 : t;
  }

  void rel(const double pos[3], double X[3]) const {
    for (int ax = 0; ax < 3; ++ax) X[ax] = pos[ax] - Xc[ax];
  }

  void loc(int c, int i, int j, int k, double pos[3]) const {
    pos[0] = i + 0.5 * kHalf[c][0];
    pos[1] = j + 0.5 * kHalf[c][1];
    pos[2] = k + 0.5 * kHalf[c][2];
  }

  // The metric used to convert between field components at a lattice point (A15).
  void field_metric(const double pos[3], double g[4][4]) const {
    double X[3];
    rel(pos, X);
    KerrFK<double> kf = kerr_fk<double>(X, cfg.m, cfg.a);
    if (kf.flat || kf.r < r_exc) {
      flat_metric(g);
      return;
    }
    metric_at(X, cfg.m, cfg.a, g);
  }

  bool excised(const double pos[3]) const {
    double X[3];
    rel(pos, X);
    KerrFK<double> kf = kerr_fk<double>(X, cfg.m, cfg.a);
    return kf.flat || kf.r < r_exc;
  }

  bool interior(int i, int j, int k) const {
    return i >= 2 && i <= n[0] - 3 && j >= 2 && j <= n[1] - 3 && k >= 2 && k <= n[2] - 3;
  }

  // Component c at the lattice point (i,j,k) of component t: mean of the nearest points of
  // c's own lattice (A7).
  double value_at(int c, int t, int i, int j, int k) const {
    const int id3[3] = {i, j, k};
    int lo[3], hi[3];
    for (int ax = 0; ax < 3; ++ax) {
      if (kHalf[c][ax] == kHalf[t][ax]) {
        lo[ax] = hi[ax] = id3[ax];
      } else if (kHalf[t][ax] == 1) {
        lo[ax] = id3[ax];
        hi[ax] = id3[ax] + 1;
      } else {
        lo[ax] = id3[ax] - 1;
        hi[ax] = id3[ax];
      }
    }
    double s = 0.0;
    int cnt = 0;
    for (int kk = lo[2]; kk <= hi[2]; ++kk)
      for (int jj = lo[1]; jj <= hi[1]; ++jj)
        for (int ii = lo[0]; ii <= hi[0]; ++ii) {
          s += F[c][idx(ii, jj, kk)];
          ++cnt;
        }
    return s / cnt;
  }

  // Full field tensor at the lattice point (i,j,k) of component t.
  void tensor_at_lattice(int t, int i, int j, int k, double Fu[4][4], double Fd[4][4]) const {
    double pos[3], g[4][4], b[3], d[3];
    loc(t, i, j, k, pos);
    field_metric(pos, g);
    for (int q = 0; q < 3; ++q) {
      d[q] = value_at(q, t, i, j, k);
      b[q] = value_at(3 + q, t, i, j, k);
    }
    complete_tensor(g, b, d, Fu, Fd);
  }

  bool literal() const { return (cfg.flags & ORC_LITERAL_HALF_STEPS) != 0; }

  // --- A23: absorbing layers -----------------------------------------------------------------
  bool layers() const { return cfg.absorb_inner > 0.0 || cfg.absorb_outer > 0.0; }

  // The fields just set become the layers' target.
  void snapshot_target() {
    if (!layers()) return;
    for (int c = 0; c < 6; ++c) F0[c] = F[c];
  }

  // Relaxation per step at the lattice point (i,j,k) of component c: the larger of the inner
  // layer's absorb_inner (r_abs - r) / (r_abs - r_exc) for r_exc <= r < r_abs and the outer
  // layer's absorb_outer ((W + 1 - s) / W)^2 for s <= W, where s - 1 counts the cells between the
  // point's cell and the outer two (frozen) index layers along the nearest axis direction.
  double absorb_kappa(int c, int i, int j, int k) const {
    double kap = 0.0;
    if (cfg.absorb_outer > 0.0) {
      const int id3[3] = {i, j, k};
      int s = n[0];
      for (int ax = 0; ax < 3; ++ax) s = std::min(s, 1 + std::min(id3[ax] - 2, n[ax] - 3 - id3[ax]));
      if (s >= 1 && s <= w_out) {
        const double u = double(w_out + 1 - s) / double(w_out);
        kap = cfg.absorb_outer * u * u;
      }
    }
    if (cfg.absorb_inner > 0.0 && r_abs > r_exc) {
      double pos[3], X[3];
      loc(c, i, j, k, pos);
      rel(pos, X);
      const KerrFK<double> kf = kerr_fk<double>(X, cfg.m, cfg.a);
      if (!kf.flat && kf.r >= r_exc && kf.r < r_abs)
        kap = std::max(kap, cfg.absorb_inner * (r_abs - kf.r) / (r_abs - r_exc));
    }
    return kap;
  }

  // v <- F0 + (1 - kappa)(v - F0) at an advanced point of component c.
  void relax(int c, int i, int j, int k, double& v) const {
    const double kap = absorb_kappa(c, i, j, k);
    if (kap > 0.0) {
      const double t = F0[c][idx(i, j, k)];
      v = t + (1.0 - kap) * (v - t);
    }
  }

  // --- Sec. 3.1: magnetic half-steps (Eqs. 9-10, time levels A21) --------------------------
  // which = 0: first half-step (b^{n-1/2} -> b^n), 1: second half-step (-> b^{n+1/2}).
  void b_half(int which) {
    const double dx4 = cfg.c * cfg.dt;
    if (!literal() && which == 0)
      for (int q = 0; q < 3; ++q) Fprev[q] = F[3 + q];
    std::vector<double> e[3];
    for (int c = 0; c < 3; ++c) e[c].assign(ncell, 0.0);
    // covariant F_{c4} at the F^{c4} lattice points
    const int nt = nthreads();
    (void)nt;
    for (int c = 0; c < 3; ++c)
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
      for (int k = 1; k <= n[2] - 2; ++k)
        for (int j = 1; j <= n[1] - 2; ++j)
          for (int i = 1; i <= n[0] - 2; ++i) {
            double Fu[4][4], Fd[4][4];
            tensor_at_lattice(c, i, j, k, Fu, Fd);
            e[c][idx(i, j, k)] = Fd[c][3];
          }
    for (int q = 0; q < 3; ++q) {
      const int al = kPair[q][0], be = kPair[q][1];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
      for (int k = 2; k <= n[2] - 3; ++k)
        for (int j = 2; j <= n[1] - 3; ++j)
          for (int i = 2; i <= n[0] - 3; ++i) {
            double pos[3];
            loc(3 + q, i, j, k, pos);
            if (excised(pos)) continue;
            const int id3[3] = {i, j, k};
            int pa[3] = {i, j, k}, pb[3] = {i, j, k};
            pa[al] += 1;
            pb[be] += 1;
            (void)id3;
            // (F_{b4}(x + e_a) - F_{b4}(x)) / dx^a + (F_{4a}(x + e_b) - F_{4a}(x)) / dx^b, dx^a = 1
            const double t1 = e[be][idx(pa[0], pa[1], pa[2])] - e[be][idx(i, j, k)];
            const double t2 = -(e[al][idx(pb[0], pb[1], pb[2])] - e[al][idx(i, j, k)]);
            const size_t id = idx(i, j, k);
            if (literal() || which == 0)
              F[3 + q][id] -= (t1 + t2) * dx4 / 2.0;
            else
              F[3 + q][id] = Fprev[q][id] - (t1 + t2) * dx4;
            if (which == 1 && layers()) relax(3 + q, i, j, k, F[3 + q][id]);
          }
    }
  }

  // Contravariant F^{jk} at the face lattice points from the current (b, d).
  void contra_h(std::vector<double> h[3]) const {
    const int nt = nthreads();
    (void)nt;
    for (int q = 0; q < 3; ++q) h[q].assign(ncell, 0.0);
    for (int q = 0; q < 3; ++q)
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
      for (int k = 1; k <= n[2] - 2; ++k)
        for (int j = 1; j <= n[1] - 2; ++j)
          for (int i = 1; i <= n[0] - 2; ++i) {
            double Fu[4][4], Fd[4][4];
            tensor_at_lattice(3 + q, i, j, k, Fu, Fd);
            h[q][idx(i, j, k)] = Fu[kPair[q][0]][kPair[q][1]];
          }
  }

  // out^a = F^{a4} + coef (4 pi/c J^a - Gamma terms - d_nu F^{a nu}) at the advanced lattice
  // points (Eq. 12 with readings A6, A8, A9); elsewhere out = F^{a4}.  Gamma terms use the
  // tensor of the current state.
  void e_update(const std::vector<double> h[3], double coef, std::vector<double> out[3]) {
    const int nt = nthreads();
    (void)nt;
    for (int al = 0; al < 3; ++al) out[al] = F[al];
    double gmax = 0.0, gscale = 0.0;
    for (int al = 0; al < 3; ++al)
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nt) reduction(max : gmax, gscale)
#endif
      for (int k = 2; k <= n[2] - 3; ++k)
        for (int j = 2; j <= n[1] - 3; ++j)
          for (int i = 2; i <= n[0] - 3; ++i) {
            double pos[3];
            loc(al, i, j, k, pos);
            if (excised(pos)) continue;
            double div = 0.0;
            for (int nu = 0; nu < 3; ++nu) {
              if (nu == al) continue;
              const int q = 3 - al - nu;
              const double sgn = (kPair[q][0] == al) ? 1.0 : -1.0;  // F^{al nu} = +-h_q
              int pm[3] = {i, j, k};
              pm[nu] -= 1;
              div += sgn * (h[q][idx(i, j, k)] - h[q][idx(pm[0], pm[1], pm[2])]);
            }
            double gterm = 0.0;
            if (!(cfg.flags & ORC_NO_GAMMA_TERMS)) {
              double X[3], G[4][4][4], Fu[4][4], Fd[4][4];
              rel(pos, X);
              christoffel_at(X, cfg.m, cfg.a, G);
              tensor_at_lattice(al, i, j, k, Fu, Fd);
              double t1 = 0.0, t2 = 0.0, scale = 0.0;
              for (int ga = 0; ga < 4; ++ga)
                for (int be = 0; be < 4; ++be) {
                  t1 += G[al][ga][be] * Fu[ga][be];
                  t2 += G[be][be][ga] * Fu[al][ga];
                  scale += std::fabs(G[al][ga][be] * Fu[ga][be]) + std::fabs(G[be][be][ga] * Fu[al][ga]);
                }
              gterm = t1 + t2;
              gmax = std::max(gmax, std::fabs(gterm));
              gscale = std::max(gscale, scale);
            }
            const size_t id = idx(i, j, k);
            out[al][id] = F[al][id] + (4.0 * kPi / cfg.c * J[al][id] - gterm - div) * coef;
          }
    gterm_max = std::max(gterm_max, gmax);
    gterm_scale = std::max(gterm_scale, gscale);
  }

  // --- Sec. 3.2: electric full step (Eqs. 11-12, readings A6, A8, A9, A21) ------------------
  void e_step() {
    const double dx4 = cfg.c * cfg.dt;
    std::vector<double> h[3], newd[3];
    contra_h(h);
    if (!literal()) {
      // midpoint predictor d* = d + (dx4/2) rhs, then the tensor at (b, d*)
      std::vector<double> dstar[3];
      e_update(h, dx4 / 2.0, dstar);
      std::vector<double> dn[3];
      for (int al = 0; al < 3; ++al) {
        dn[al] = F[al];
        F[al] = dstar[al];
      }
      contra_h(h);
      for (int al = 0; al < 3; ++al) F[al].swap(dn[al]);
    }
    e_update(h, dx4, newd);
    if (layers())
      for (int al = 0; al < 3; ++al)
        for (int k = 2; k <= n[2] - 3; ++k)
          for (int j = 2; j <= n[1] - 3; ++j)
            for (int i = 2; i <= n[0] - 3; ++i) {
              double pos[3];
              loc(al, i, j, k, pos);
              if (!excised(pos)) relax(al, i, j, k, newd[al][idx(i, j, k)]);
            }
    for (int al = 0; al < 3; ++al) F[al].swap(newd[al]);
  }

  // CIC gather of component c at grid position x (Sec. 3.3; weights trilinear, reading A5).
  bool gather(int c, const double x[3], double* out) const {
    int i0[3];
    double w[3];
    for (int ax = 0; ax < 3; ++ax) {
      const double s = x[ax] - 0.5 * kHalf[c][ax];
      if (!(s >= 0.0) || !(s <= n[ax] - 1)) return false;
      i0[ax] = (int)std::floor(s);
      if (i0[ax] > n[ax] - 2) i0[ax] = n[ax] - 2;
      w[ax] = s - i0[ax];
    }
    double sum = 0.0;
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const double W = (di ? w[0] : 1.0 - w[0]) * (dj ? w[1] : 1.0 - w[1]) * (dk ? w[2] : 1.0 - w[2]);
          sum += W * F[c][idx(i0[0] + di, i0[1] + dj, i0[2] + dk)];
        }
    *out = sum;
    return true;
  }

  // Eq. 15: a~^a = (q/m) F^a_b u^b - Gamma^a_{mn} u^m u^n at (x, u).
  bool accel(const double x[4], const double u[4], double qm, double out[4]) const {
    double X[3];
    rel(x, X);
    double g[4][4], G[4][4][4];
    metric_at(X, cfg.m, cfg.a, g);
    christoffel_at(X, cfg.m, cfg.a, G);
    double Fu[4][4], Fd[4][4];
    if (cfg.flags & ORC_ANALYTIC_WALD) {
      // the field tensor evaluated in closed form at the particle instead of gathered
      wald_field(X, cfg.m, cfg.a, wald_B0, Fd, Fu);
    } else {
      double b[3], d[3];
      for (int q = 0; q < 3; ++q) {
        if (!gather(q, x, &d[q])) return false;
        if (!gather(3 + q, x, &b[q])) return false;
      }
      complete_tensor(g, b, d, Fu, Fd);
    }
    for (int al = 0; al < 4; ++al) {
      double lor = 0.0;
      for (int be = 0; be < 4; ++be) {
        double mix = 0.0;  // F^a_b = F^{ac} g_{cb}
        for (int ga = 0; ga < 4; ++ga) mix += Fu[al][ga] * g[ga][be];
        lor += mix * u[be];
      }
      double grav = 0.0;
      for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) grav += G[al][mu][nu] * u[mu] * u[nu];
      out[al] = qm * lor - grav;
    }
    return true;
  }

  // Eq. 18 over [Is, If] x [Js, Jf] in the plane x^K = xK, Q x Q Gauss-Legendre.
  double area(int K, double xK, int I, double Is, double If, int Jx, double Js, double Jf) const {
    const int Q = (int)glx.size();
    double s = 0.0;
    for (int p = 0; p < Q; ++p)
      for (int q = 0; q < Q; ++q) {
        double pos[3];
        pos[K] = xK;
        pos[I] = 0.5 * (Is + If) + 0.5 * (If - Is) * glx[p];
        pos[Jx] = 0.5 * (Js + Jf) + 0.5 * (Jf - Js) * glx[q];
        double X[3], g[4][4];
        rel(pos, X);
        metric_at(X, cfg.m, cfg.a, g);
        const double integrand = std::sqrt(g[I][I] * g[Jx][Jx] - g[I][Jx] * g[I][Jx]);
        s += glw[p] * glw[q] * integrand;
      }
    return s * 0.25 * (If - Is) * (Jf - Js);
  }

  // Sec. 4 surface weights for flux in direction K through the face of `cell`, split at
  // the transverse coordinates of P.  W[0..3] = W_{i,j}, W_{i+1,j}, W_{i,j+1}, W_{i+1,j+1}.
  void face_weights(int K, const double P[3], const int cell[3], double W[4]) const {
    const int I = (K + 1) % 3, Jx = (K + 2) % 3;
    const double i0 = cell[I], j0 = cell[Jx];
    const double A00 = area(K, P[K], I, P[I], i0 + 1.0, Jx, P[Jx], j0 + 1.0);
    const double A10 = area(K, P[K], I, i0, P[I], Jx, P[Jx], j0 + 1.0);
    const double A01 = area(K, P[K], I, P[I], i0 + 1.0, Jx, j0, P[Jx]);
    const double A11 = area(K, P[K], I, i0, P[I], Jx, j0, P[Jx]);
    const double FA = A00 + A10 + A01 + A11;
    W[0] = A00 / FA;
    W[1] = A10 / FA;
    W[2] = A01 / FA;
    W[3] = A11 / FA;
  }

  // Sec. 4: Umeda zig-zag split of x1 -> x2 into two segments, flux through the faces of
  // each segment's cell with the curved surface weights, J = rho gamma v (A13).
  bool deposit(const double x1[3], const double x2[3], double qmacro, double gbar, std::vector<double>* Jt) const {
    int c1[3], c2[3];
    double xr[3];
    for (int ax = 0; ax < 3; ++ax) {
      c1[ax] = (int)std::floor(x1[ax]);
      c2[ax] = (int)std::floor(x2[ax]);
      const double mid = 0.5 * (x1[ax] + x2[ax]);
      xr[ax] = std::min((double)std::min(c1[ax], c2[ax]) + 1.0, std::max((double)std::max(c1[ax], c2[ax]), mid));
    }
    for (int ax = 0; ax < 3; ++ax)
      if (c1[ax] < 0 || c2[ax] < 0 || c1[ax] > n[ax] - 2 || c2[ax] > n[ax] - 2) return false;
    const double* segs[2][2] = {{x1, xr}, {xr, x2}};
    const int* cells[2] = {c1, c2};
    for (int s = 0; s < 2; ++s) {
      const double* a = segs[s][0];
      const double* b = segs[s][1];
      const int* cell = cells[s];
      double P[3];
      for (int ax = 0; ax < 3; ++ax) P[ax] = 0.5 * (a[ax] + b[ax]);
      for (int K = 0; K < 3; ++K) {
        const double flux = qmacro * gbar * (b[K] - a[K]) / cfg.dt;
        double W[4];
        face_weights(K, P, cell, W);
        const int I = (K + 1) % 3, Jx = (K + 2) % 3;
        for (int dj = 0; dj < 2; ++dj)
          for (int di = 0; di < 2; ++di) {
            int node[3];
            node[K] = cell[K];
            node[I] = cell[I] + di;
            node[Jx] = cell[Jx] + dj;
            Jt[K][idx(node[0], node[1], node[2])] += flux * W[dj * 2 + di];
          }
      }
    }
    return true;
  }

  // Sec. 3.3: RK4 step of one particle (reading A1), deposit, removal flag.
  // Returns ORC_OK, or an error code.
  int push_deposit_one(Species& s, size_t p, std::vector<double>* Jt, bool* remove, bool* horizon,
                       long long* fallbacks) const {
    const double c = cfg.c, dt = cfg.dt;
    double x0[4], u0[4];
    for (int al = 0; al < 4; ++al) {
      x0[al] = s.x[al][p];
      u0[al] = s.u[al][p];
    }
    double x1[4], u1[4];
    if (cfg.flags & ORC_RK4_AS_PRINTED) {
      const int e = rk4_as_printed(x0, u0, s.qm, fallbacks, x1, u1);
      if (e != ORC_OK) return e;
      return finish_push(s, p, x0, x1, u1, Jt, remove, horizon);
    }
    double k1u[4], k2u[4], k3u[4], k4u[4];
    double k1x[4], k2x[4], k3x[4], k4x[4];
    if (!accel(x0, u0, s.qm, k1u)) return ORC_ERR_CFL;
    int fb = 0;
    const double g1 = gamma_f(u0[3], k1u[3], c, dt, &fb);  // Eq. 16 at (x_n, u_n)
    *fallbacks += fb;
    const double h = dt / g1;
    double xs[4], us[4];
    for (int al = 0; al < 4; ++al) k1x[al] = u0[al];
    for (int al = 0; al < 4; ++al) {
      xs[al] = x0[al] + 0.5 * h * k1x[al];
      us[al] = u0[al] + 0.5 * h * k1u[al];
    }
    for (int al = 0; al < 4; ++al) k2x[al] = us[al];
    if (!accel(xs, us, s.qm, k2u)) return ORC_ERR_CFL;
    for (int al = 0; al < 4; ++al) {
      xs[al] = x0[al] + 0.5 * h * k2x[al];
      us[al] = u0[al] + 0.5 * h * k2u[al];
    }
    for (int al = 0; al < 4; ++al) k3x[al] = us[al];
    if (!accel(xs, us, s.qm, k3u)) return ORC_ERR_CFL;
    for (int al = 0; al < 4; ++al) {
      xs[al] = x0[al] + h * k3x[al];
      us[al] = u0[al] + h * k3u[al];
    }
    for (int al = 0; al < 4; ++al) k4x[al] = us[al];
    if (!accel(xs, us, s.qm, k4u)) return ORC_ERR_CFL;
    for (int al = 0; al < 4; ++al) {
      x1[al] = x0[al] + h / 6.0 * (k1x[al] + 2.0 * k2x[al] + 2.0 * k3x[al] + k4x[al]);
      u1[al] = u0[al] + h / 6.0 * (k1u[al] + 2.0 * k2u[al] + 2.0 * k3u[al] + k4u[al]);
    }
    return finish_push(s, p, x0, x1, u1, Jt, remove, horizon);
  }

  // The RK4 steps of Sec. 3.3 as printed, for the ablation (ORC_RK4_AS_PRINTED).  Stage k has
  // the trapezoid velocity ut_k = (u_n + u_k)/2 (ut_1 = u_n), position x_n + ut_k dtau_{k-1}, the
  // acceleration a_k = a~(x_k, ut_k) and gamma_k = f(ut_k^4, a_k^4) (Eq. 16); u_{k+1} = u_n + a_k
  // dtau_k; dtau_1 = dt/(2 gamma_1), dtau_2 = dt/gamma_2, dtau_3 = dt/gamma_3,
  // dtau_4 = dt/(2 gamma_4).  The final sums are taken as increments of x_n and u_n.
  int rk4_as_printed(const double x0[4], const double u0[4], double qm, long long* fallbacks, double x1[4],
                     double u1[4]) const {
    const double dt = cfg.dt, c = cfg.c;
    double ut[4][4], a[4][4], dtau[4];
    double xk[4], uk[4];
    for (int k = 0; k < 4; ++k) {
      for (int al = 0; al < 4; ++al) {
        if (k == 0) {
          ut[k][al] = u0[al];
          xk[al] = x0[al];
        } else {
          uk[al] = u0[al] + a[k - 1][al] * dtau[k - 1];
          ut[k][al] = 0.5 * (u0[al] + uk[al]);
        }
      }
      if (k > 0)
        for (int al = 0; al < 4; ++al) xk[al] = x0[al] + ut[k][al] * dtau[k - 1];
      if (!accel(xk, ut[k], qm, a[k])) return ORC_ERR_CFL;
      int fb = 0;
      const double g = gamma_f(ut[k][3], a[k][3], c, dt, &fb);
      *fallbacks += fb;
      dtau[k] = (k == 0 || k == 3) ? dt / (2.0 * g) : dt / g;
    }
    for (int al = 0; al < 4; ++al) {
      x1[al] = x0[al] + (ut[0][al] * dtau[0] + 2.0 * (ut[1][al] * dtau[1] + ut[2][al] * dtau[2]) +
                         ut[3][al] * dtau[3]) / 6.0;
      u1[al] = u0[al] + (a[0][al] * dtau[0] + 2.0 * (a[1][al] * dtau[1] + a[2][al] * dtau[2]) +
                         a[3][al] * dtau[3]) / 6.0;
    }
    return ORC_OK;
  }

  // After the RK4 step: checks, deposit of x_n -> x_{n+1}, new state, removal flag.
  int finish_push(Species& s, size_t p, const double x0[4], const double x1[4], const double u1[4],
                  std::vector<double>* Jt, bool* remove, bool* horizon) const {
    const double c = cfg.c;
    const double u0_4 = s.u[3][p];
    for (int al = 0; al < 4; ++al)
      if (!std::isfinite(x1[al]) || !std::isfinite(u1[al])) return ORC_ERR_NONFINITE;
    for (int ax = 0; ax < 3; ++ax)
      if (std::fabs(x1[ax] - x0[ax]) >= 1.0) return ORC_ERR_CFL;
    const double gbar = (cfg.flags & ORC_NO_GAMMA_IN_J) ? 1.0 : (u0_4 + u1[3]) / (2.0 * c);
    if (s.qmacro != 0.0)
      if (!deposit(x0, x1, s.qmacro, gbar, Jt)) return ORC_ERR_CFL;
    for (int al = 0; al < 4; ++al) {
      s.x[al][p] = x1[al];
      s.u[al][p] = u1[al];
    }
    double X[3];
    rel(x1, X);
    const KerrFK<double> kf = kerr_fk<double>(X, cfg.m, cfg.a);
    *horizon = (cfg.m > 0.0) && (kf.flat || kf.r <= r_plus);
    bool outer = false;
    for (int ax = 0; ax < 3; ++ax)
      if (x1[ax] < 1.0 || x1[ax] > n[ax] - 2) outer = true;
    *remove = *horizon || outer;
    return ORC_OK;
  }

  int push_deposit_all() {
    const int nthreads = this->nthreads();
    int err = ORC_OK;
    for (auto& s : sp) {
      const size_t np = s.id.size();
      for (int ax = 0; ax < 3; ++ax) s.last_x0[ax] = s.x[ax];
      s.last_id = s.id;
      std::vector<char> rem(np, 0), hor(np, 0);
      std::vector<std::vector<double>> Jt((size_t)nthreads * 3);
      for (auto& v : Jt) v.assign(ncell, 0.0);
      std::vector<int> terr(nthreads, ORC_OK);
      std::vector<long long> tfb(nthreads, 0);
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
      {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        const size_t lo = np * (size_t)t / nthreads, hi = np * (size_t)(t + 1) / nthreads;
        for (size_t p = lo; p < hi; ++p) {
          bool r = false, hz = false;
          const int e = push_deposit_one(s, p, &Jt[(size_t)t * 3], &r, &hz, &tfb[t]);
          if (e != ORC_OK) {
            terr[t] = e;
            break;
          }
          rem[p] = r;
          hor[p] = hz;
        }
      }
      for (int ax = 0; ax < 3; ++ax) s.last_x1[ax] = s.x[ax];
      for (int t = 0; t < nthreads; ++t) {
        if (terr[t] != ORC_OK && err == ORC_OK) err = terr[t];
        stat_fallback += tfb[t];
        for (int K = 0; K < 3; ++K)
          for (size_t i = 0; i < ncell; ++i) J[K][i] += Jt[(size_t)t * 3 + K][i];
      }
      // removal (A15), keeping id order
      size_t w = 0;
      for (size_t p = 0; p < np; ++p) {
        if (rem[p]) {
          if (hor[p])
            ++stat_removed_horizon;
          else
            ++stat_removed_outer;
          continue;
        }
        for (int al = 0; al < 4; ++al) {
          s.x[al][w] = s.x[al][p];
          s.u[al][w] = s.u[al][p];
        }
        s.id[w] = s.id[p];
        ++w;
      }
      for (int al = 0; al < 4; ++al) {
        s.x[al].resize(w);
        s.u[al].resize(w);
      }
      s.id.resize(w);
      if (err != ORC_OK) return err;
    }
    return err;
  }

  void zero_j() {
    for (int K = 0; K < 3; ++K) std::fill(J[K].begin(), J[K].end(), 0.0);
  }

  // Sec. 2.2 cycle: B half-step, push + deposit, B half-step, E step.
  int step() {
    const bool fields = !(cfg.flags & ORC_FROZEN_FIELDS);
    if (fields) b_half(0);
    zero_j();
    const int e = push_deposit_all();
    if (e != ORC_OK) return e;
    if (fields) {
      b_half(1);
      e_step();
    }
    ++stat_steps;
    return ORC_OK;
  }
};

// Future-directed completion of a 4-velocity with g_mn u^m u^n = -c^2.
// mode 1: usp are the covariant spatial components u_i; mode 2: contravariant u^i.
int solve_u4(const double X[3], double m, double a, double c, const double usp[3], int mode, double u[4]) {
  double g[4][4], gi[4][4];
  metric_at(X, m, a, g);
  if (!invert4(g, gi)) return ORC_ERR_INVALID;
  if (mode == 1) {
    // g^{44} u_4^2 + 2 g^{4i} u_i u_4 + (g^{ij} u_i u_j + c^2) = 0, g^{44} < 0
    const double A = gi[3][3];
    double B = 0.0, C = c * c;
    for (int i = 0; i < 3; ++i) {
      B += 2.0 * gi[3][i] * usp[i];
      for (int j = 0; j < 3; ++j) C += gi[i][j] * usp[i] * usp[j];
    }
    const double disc = B * B - 4.0 * A * C;
    if (!(A < 0.0) || disc < 0.0) return ORC_ERR_INVALID;
    const double r1 = (-B + std::sqrt(disc)) / (2.0 * A), r2 = (-B - std::sqrt(disc)) / (2.0 * A);
    double ul[4] = {usp[0], usp[1], usp[2], 0.0};
    int found = 0;
    for (double cand : {r1, r2}) {
      ul[3] = cand;
      double u4 = 0.0;
      for (int nu = 0; nu < 4; ++nu) u4 += gi[3][nu] * ul[nu];
      if (u4 > 0.0 && !found) {
        for (int mu = 0; mu < 4; ++mu) {
          double s = 0.0;
          for (int nu = 0; nu < 4; ++nu) s += gi[mu][nu] * ul[nu];
          u[mu] = s;
        }
        found = 1;
      }
    }
    return found ? ORC_OK : ORC_ERR_INVALID;
  }
  if (mode == 2) {
    // g_44 (u^4)^2 + 2 g_4i u^i u^4 + (g_ij u^i u^j + c^2) = 0; unique positive root needs g_44 < 0
    const double A = g[3][3];
    double B = 0.0, C = c * c;
    for (int i = 0; i < 3; ++i) {
      B += 2.0 * g[3][i] * usp[i];
      for (int j = 0; j < 3; ++j) C += g[i][j] * usp[i] * usp[j];
    }
    const double disc = B * B - 4.0 * A * C;
    if (!(A < 0.0) || disc < 0.0) return ORC_ERR_INVALID;
    const double r1 = (-B + std::sqrt(disc)) / (2.0 * A), r2 = (-B - std::sqrt(disc)) / (2.0 * A);
    const double u4 = std::max(r1, r2);
    if (!(u4 > 0.0)) return ORC_ERR_INVALID;
    u[0] = usp[0];
    u[1] = usp[1];
    u[2] = usp[2];
    u[3] = u4;
    return ORC_OK;
  }
  return ORC_ERR_INVALID;
}

// Wald's stationary vacuum field: A_m = (B0/2) (xi_phi + 2 a xi_t)_m with the rotation
// Killing vector xi_phi = x d_y - y d_x and xi_t = d_4; F_mn = d_m A_n - d_n A_m.
void wald_field(const double X[3], double m, double a, double B0, double Fd[4][4], double Fu[4][4]) {
  Dual Xd[3];
  for (int i = 0; i < 3; ++i) {
    Xd[i] = Dual(X[i]);
    Xd[i].d[i] = 1.0;
  }
  Dual g[4][4];
  kerr_metric<Dual>(Xd, m, a, g);
  Dual xi[4] = {-Xd[1], Xd[0], Dual(0.0), Dual(2.0 * a)};
  Dual A[4];
  for (int mu = 0; mu < 4; ++mu) {
    A[mu] = Dual(0.0);
    for (int nu = 0; nu < 4; ++nu) A[mu] = A[mu] + g[mu][nu] * xi[nu];
    A[mu] = A[mu] * (0.5 * B0);
  }
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      const double dmAn = (mu < 3) ? A[nu].d[mu] : 0.0;
      const double dnAm = (nu < 3) ? A[mu].d[nu] : 0.0;
      Fd[mu][nu] = dmAn - dnAm;
    }
  double gv[4][4], gi[4][4];
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) gv[mu][nu] = g[mu][nu].v;
  invert4(gv, gi);
  lower2(gi, Fd, Fu);  // raising uses the same contraction with g^{-1}
}

void to16(const double A[4][4], double* o) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) o[i * 4 + j] = A[i][j];
}
void from16(const double* o, double A[4][4]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) A[i][j] = o[i * 4 + j];
}

}  // namespace

// =======================================================================================
// C ABI used by the Python wrapper (oracle/__init__.py).
// =======================================================================================
extern "C" {

double orc_kerr_r(const double* X, double a) {
  return kerr_fk<double>(X, 0.0, a).r;
}

void orc_kerr_fk(const double* X, double m, double a, double* out6) {
  KerrFK<double> kf = kerr_fk<double>(X, m, a);
  out6[0] = kf.r;
  out6[1] = kf.f;
  for (int i = 0; i < 4; ++i) out6[2 + i] = kf.k[i];
}

void orc_metric(const double* X, double m, double a, double* g16) {
  double g[4][4];
  metric_at(X, m, a, g);
  to16(g, g16);
}

int orc_metric_inverse(const double* X, double m, double a, double* gi16) {
  double g[4][4], gi[4][4];
  metric_at(X, m, a, g);
  if (!invert4(g, gi)) return ORC_ERR_INVALID;
  to16(gi, gi16);
  return ORC_OK;
}

double orc_metric_det(const double* X, double m, double a) {
  double g[4][4];
  metric_at(X, m, a, g);
  return det4(g);
}

void orc_metric_grad(const double* X, double m, double a, double* dg48) {
  double g[4][4], dg[4][4][4];
  metric_grad(X, m, a, g, dg);
  for (int l = 0; l < 3; ++l)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = 0; nu < 4; ++nu) dg48[(l * 4 + mu) * 4 + nu] = dg[l][mu][nu];
}

void orc_christoffel(const double* X, double m, double a, double* G64) {
  double G[4][4][4];
  christoffel_at(X, m, a, G);
  for (int al = 0; al < 4; ++al)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = 0; nu < 4; ++nu) G64[(al * 4 + mu) * 4 + nu] = G[al][mu][nu];
}

// Eq. 7: gamma^-2 = -g_ij v^i v^j / c^2 with v^4 = c (indices over 1..4).
double orc_gamma_from_v(const double* X, double m, double a, double c, const double* v3) {
  double g[4][4];
  metric_at(X, m, a, g);
  const double v[4] = {v3[0], v3[1], v3[2], c};
  double s = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) s += g[i][j] * v[i] * v[j];
  const double inv2 = -s / (c * c);
  return inv2 > 0.0 ? 1.0 / std::sqrt(inv2) : NAN;
}

double orc_gamma_f(double u4, double a4, double c, double dt, int* fallback) {
  return gamma_f(u4, a4, c, dt, fallback);
}

int orc_solve_u4(const double* X, double m, double a, double c, const double* usp, int mode, double* u4out) {
  return solve_u4(X, m, a, c, usp, mode, u4out);
}

int orc_complete_tensor(const double* g16, const double* b3, const double* d3, double* Fu16, double* Fd16) {
  double g[4][4], Fu[4][4], Fd[4][4];
  from16(g16, g);
  if (!complete_tensor(g, b3, d3, Fu, Fd)) return ORC_ERR_INVALID;
  to16(Fu, Fu16);
  to16(Fd, Fd16);
  return ORC_OK;
}

void orc_gauss_legendre(int Q, double* x, double* w) {
  std::vector<double> gx, gw;
  gauss_legendre(Q, gx, gw);
  for (int i = 0; i < Q; ++i) {
    x[i] = gx[i];
    w[i] = gw[i];
  }
}

// Sec. 3.3 sub-volume weights taken literally: VOLUME(...) = integral of sqrt(-det g) by
// Q^3 Gauss-Legendre per sub-box.  P is the particle's grid position, cell its cell,
// Xc the centre of mass; W in the order of the paper's list (i,j,k), (i+1,j,k), (i,j+1,k),
// (i,j,k+1), (i+1,j+1,k), (i,j+1,k+1), (i+1,j,k+1), (i+1,j+1,k+1).
void orc_volume_weights(const double* P, const int* cell, const double* Xc, double m, double a, int Q, double* W8) {
  std::vector<double> gx, gw;
  gauss_legendre(Q, gx, gw);
  auto volume = [&](double x0, double x1, double y0, double y1, double z0, double z1) {
    double s = 0.0;
    for (int p = 0; p < Q; ++p)
      for (int q = 0; q < Q; ++q)
        for (int r = 0; r < Q; ++r) {
          const double X[3] = {0.5 * (x0 + x1) + 0.5 * (x1 - x0) * gx[p] - Xc[0],
                               0.5 * (y0 + y1) + 0.5 * (y1 - y0) * gx[q] - Xc[1],
                               0.5 * (z0 + z1) + 0.5 * (z1 - z0) * gx[r] - Xc[2]};
          double g[4][4];
          metric_at(X, m, a, g);
          s += gw[p] * gw[q] * gw[r] * std::sqrt(-det4(g));
        }
    return s * 0.125 * (x1 - x0) * (y1 - y0) * (z1 - z0);
  };
  const double xi = cell[0], yj = cell[1], zk = cell[2];
  const double cellv = volume(xi, xi + 1, yj, yj + 1, zk, zk + 1);
  const double xp = P[0], yp = P[1], zp = P[2];
  W8[0] = volume(xp, xi + 1, yp, yj + 1, zp, zk + 1) / cellv;
  W8[1] = volume(xi, xp, yp, yj + 1, zp, zk + 1) / cellv;
  W8[2] = volume(xp, xi + 1, yj, yp, zp, zk + 1) / cellv;
  W8[3] = volume(xp, xi + 1, yp, yj + 1, zk, zp) / cellv;
  W8[4] = volume(xi, xp, yj, yp, zp, zk + 1) / cellv;
  W8[5] = volume(xp, xi + 1, yj, yp, zk, zp) / cellv;
  W8[6] = volume(xi, xp, yp, yj + 1, zk, zp) / cellv;
  W8[7] = volume(xi, xp, yj, yp, zk, zp) / cellv;
}

void orc_wald_field(const double* X, double m, double a, double B0, double* Fd16, double* Fu16) {
  double Fd[4][4], Fu[4][4];
  wald_field(X, m, a, B0, Fd, Fu);
  to16(Fd, Fd16);
  to16(Fu, Fu16);
}

void* orc_create(const orc_config* cfg) {
  if (!cfg || cfg->nx < 6 || cfg->ny < 6 || cfg->nz < 6 || !(cfg->dt > 0) || !(cfg->c > 0) || cfg->m < 0 ||
      std::fabs(cfg->a) > cfg->m || cfg->quad_order < 1 || cfg->quad_order > 16)
    return nullptr;
  Ctx* ctx = new Ctx();
  ctx->cfg = *cfg;
  ctx->n[0] = cfg->nx;
  ctx->n[1] = cfg->ny;
  ctx->n[2] = cfg->nz;
  for (int ax = 0; ax < 3; ++ax) ctx->Xc[ax] = 0.5 * (ctx->n[ax] - 1);
  // A24: a slab of a larger run keeps the run's centre
  const int nz_total = cfg->nz_total > 0 ? cfg->nz_total : cfg->nz;
  const bool slab = cfg->z_origin != 0 || nz_total != cfg->nz;
  if (cfg->z_origin < 0 || cfg->z_origin + cfg->nz > nz_total || (slab && cfg->absorb_outer > 0.0)) {
    delete ctx;
    return nullptr;
  }
  ctx->Xc[2] = 0.5 * (nz_total - 1) - cfg->z_origin;
  ctx->r_plus = cfg->m + std::sqrt(std::max(0.0, cfg->m * cfg->m - cfg->a * cfg->a));
  if (!(cfg->absorb_inner >= 0.0 && cfg->absorb_inner <= 1.0 && cfg->absorb_outer >= 0.0 &&
        cfg->absorb_outer <= 1.0)) {
    delete ctx;
    return nullptr;
  }
  ctx->r_exc = cfg->r_excise > 0 ? cfg->r_excise : (cfg->absorb_inner > 0.0 ? 0.5 : 1.0) * ctx->r_plus;
  ctx->r_abs = ctx->r_plus;
  ctx->w_out = cfg->absorb_width > 0 ? cfg->absorb_width : 8;
  ctx->ncell = (size_t)cfg->nx * cfg->ny * cfg->nz;
  for (auto& f : ctx->F) f.assign(ctx->ncell, 0.0);
  if (ctx->layers())
    for (auto& f : ctx->F0) f.assign(ctx->ncell, 0.0);
  for (auto& j : ctx->J) j.assign(ctx->ncell, 0.0);
  gauss_legendre(cfg->quad_order, ctx->glx, ctx->glw);
  return ctx;
}

void orc_destroy(void* p) { delete static_cast<Ctx*>(p); }

double orc_r_plus(void* p) { return static_cast<Ctx*>(p)->r_plus; }

int orc_set_fields(void* p, const double* d3, const double* b3) {
  Ctx* ctx = static_cast<Ctx*>(p);
  for (int q = 0; q < 3; ++q) {
    std::memcpy(ctx->F[q].data(), d3 + q * ctx->ncell, ctx->ncell * sizeof(double));
    std::memcpy(ctx->F[3 + q].data(), b3 + q * ctx->ncell, ctx->ncell * sizeof(double));
  }
  ctx->snapshot_target();
  return ORC_OK;
}

// Replace the absorbing layers' target (A23) without touching the fields.
int orc_set_absorb_target(void* p, const double* d3, const double* b3) {
  Ctx* ctx = static_cast<Ctx*>(p);
  if (!ctx->layers()) return ORC_ERR_INVALID;
  for (int q = 0; q < 3; ++q) {
    std::memcpy(ctx->F0[q].data(), d3 + q * ctx->ncell, ctx->ncell * sizeof(double));
    std::memcpy(ctx->F0[3 + q].data(), b3 + q * ctx->ncell, ctx->ncell * sizeof(double));
  }
  return ORC_OK;
}

// Relaxation per step of the absorbing layers at component c's lattice point (i, j, k) (A23).
double orc_absorb_kappa(void* p, int c, int i, int j, int k) {
  return static_cast<Ctx*>(p)->absorb_kappa(c, i, j, k);
}

int orc_set_j(void* p, const double* J3) {
  Ctx* ctx = static_cast<Ctx*>(p);
  for (int q = 0; q < 3; ++q) std::memcpy(ctx->J[q].data(), J3 + q * ctx->ncell, ctx->ncell * sizeof(double));
  return ORC_OK;
}

// Contravariant F^{jk} (h: F^{yz}, F^{zx}, F^{xy}) at the b face lattice points, from the current (b, d)
// as the E step converts them (A7); zero on the outer index layer.
int orc_get_contra_h(void* p, double* h3) {
  Ctx* ctx = static_cast<Ctx*>(p);
  std::vector<double> h[3];
  ctx->contra_h(h);
  for (int q = 0; q < 3; ++q) std::memcpy(h3 + q * ctx->ncell, h[q].data(), ctx->ncell * sizeof(double));
  return ORC_OK;
}

int orc_get_fields(void* p, double* d3, double* b3, double* J3) {
  Ctx* ctx = static_cast<Ctx*>(p);
  for (int q = 0; q < 3; ++q) {
    if (d3) std::memcpy(d3 + q * ctx->ncell, ctx->F[q].data(), ctx->ncell * sizeof(double));
    if (b3) std::memcpy(b3 + q * ctx->ncell, ctx->F[3 + q].data(), ctx->ncell * sizeof(double));
    if (J3) std::memcpy(J3 + q * ctx->ncell, ctx->J[q].data(), ctx->ncell * sizeof(double));
  }
  return ORC_OK;
}

// Uniform contravariant field (Eq. 8: F^{4j} = E^j, F^{jk} = eps^{jkl} B^l), converted to the
// prognostic components at every lattice point.
int orc_init_uniform_field(void* p, const double* E3, const double* B3) {
  Ctx* ctx = static_cast<Ctx*>(p);
  double Fu[4][4];
  const double h[3] = {B3[0], B3[1], B3[2]};
  const double d[3] = {-E3[0], -E3[1], -E3[2]};
  build_up(h, d, Fu);
  for (int c = 0; c < 6; ++c)
    for (int k = 0; k < ctx->n[2]; ++k)
      for (int j = 0; j < ctx->n[1]; ++j)
        for (int i = 0; i < ctx->n[0]; ++i) {
          double v;
          if (c < 3) {
            v = Fu[c][3];
          } else {
            double pos[3], g[4][4], Fd[4][4];
            ctx->loc(c, i, j, k, pos);
            ctx->field_metric(pos, g);
            lower2(g, Fu, Fd);
            v = Fd[kPair[c - 3][0]][kPair[c - 3][1]];
          }
          ctx->F[c][ctx->idx(i, j, k)] = v;
        }
  ctx->snapshot_target();
  return ORC_OK;
}

int orc_init_wald(void* p, double B0) {
  Ctx* ctx = static_cast<Ctx*>(p);
  for (int c = 0; c < 6; ++c)
    for (int k = 0; k < ctx->n[2]; ++k)
      for (int j = 0; j < ctx->n[1]; ++j)
        for (int i = 0; i < ctx->n[0]; ++i) {
          double pos[3], X[3], Fd[4][4], Fu[4][4];
          ctx->loc(c, i, j, k, pos);
          ctx->rel(pos, X);
          wald_field(X, ctx->cfg.m, ctx->cfg.a, B0, Fd, Fu);
          ctx->F[c][ctx->idx(i, j, k)] = (c < 3) ? Fu[c][3] : Fd[kPair[c - 3][0]][kPair[c - 3][1]];
        }
  ctx->snapshot_target();
  return ORC_OK;
}

// umode 0: u4 holds u^1..u^4; 1: planes 0..2 hold covariant u_i (u^a solved);
// 2: planes 0..2 hold contravariant u^i (u^4 solved).
int orc_load_particles(void* p, int species, double qm, double qmacro, long long n, const double* x4,
                       const double* u4, const uint32_t* ids, int umode) {
  Ctx* ctx = static_cast<Ctx*>(p);
  if (species < 0 || n < 0) return ORC_ERR_INVALID;
  if ((int)ctx->sp.size() <= species) ctx->sp.resize(species + 1);
  Species& s = ctx->sp[species];
  s.qm = qm;
  s.qmacro = qmacro;
  std::vector<size_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](size_t i, size_t j) { return ids[i] < ids[j]; });
  for (int al = 0; al < 4; ++al) {
    s.x[al].assign(n, 0.0);
    s.u[al].assign(n, 0.0);
  }
  s.id.assign(n, 0);
  long long w = 0;
  for (long long o = 0; o < n; ++o) {
    const size_t i = order[o];
    double x[4], u[4];
    for (int al = 0; al < 4; ++al) x[al] = x4[al * n + i];
    for (int ax = 0; ax < 3; ++ax)
      if (!(x[ax] >= 1.0 && x[ax] <= ctx->n[ax] - 2)) return ORC_ERR_INVALID;
    // removal rule r <= r_+ (A15) applies from the start
    if (ctx->cfg.m > 0.0) {
      double X[3];
      ctx->rel(x, X);
      const KerrFK<double> kf = kerr_fk<double>(X, ctx->cfg.m, ctx->cfg.a);
      if (kf.flat || kf.r <= ctx->r_plus) {
        ++ctx->stat_removed_horizon;
        continue;
      }
    }
    if (umode == 0) {
      for (int al = 0; al < 4; ++al) u[al] = u4[al * n + i];
    } else {
      double X[3], usp[3] = {u4[0 * n + i], u4[1 * n + i], u4[2 * n + i]};
      ctx->rel(x, X);
      const int e = solve_u4(X, ctx->cfg.m, ctx->cfg.a, ctx->cfg.c, usp, umode, u);
      if (e != ORC_OK) return e;
    }
    for (int al = 0; al < 4; ++al) {
      s.x[al][w] = x[al];
      s.u[al][w] = u[al];
    }
    s.id[w] = ids[i];
    ++w;
  }
  for (int al = 0; al < 4; ++al) {
    s.x[al].resize(w);
    s.u[al].resize(w);
  }
  s.id.resize(w);
  return ORC_OK;
}

long long orc_num_particles(void* p, int species) {
  Ctx* ctx = static_cast<Ctx*>(p);
  if (species < 0 || species >= (int)ctx->sp.size()) return 0;
  return (long long)ctx->sp[species].id.size();
}

int orc_get_particles(void* p, int species, double* x4, double* u4, uint32_t* ids) {
  Ctx* ctx = static_cast<Ctx*>(p);
  if (species < 0 || species >= (int)ctx->sp.size()) return ORC_ERR_INVALID;
  const Species& s = ctx->sp[species];
  const size_t n = s.id.size();
  for (int al = 0; al < 4; ++al)
    for (size_t i = 0; i < n; ++i) {
      if (x4) x4[al * n + i] = s.x[al][i];
      if (u4) u4[al * n + i] = s.u[al][i];
    }
  if (ids)
    for (size_t i = 0; i < n; ++i) ids[i] = s.id[i];
  return ORC_OK;
}

int orc_step(void* p, int nsteps) {
  Ctx* ctx = static_cast<Ctx*>(p);
  for (int s = 0; s < nsteps; ++s) {
    const int e = ctx->step();
    if (e != ORC_OK) return e;
  }
  return ORC_OK;
}

int orc_stage_b_half(void* p) {
  static_cast<Ctx*>(p)->b_half(0);
  return ORC_OK;
}
int orc_stage_b_half2(void* p) {
  static_cast<Ctx*>(p)->b_half(1);
  return ORC_OK;
}
int orc_stage_e(void* p) {
  static_cast<Ctx*>(p)->e_step();
  return ORC_OK;
}
int orc_stage_zero_j(void* p) {
  static_cast<Ctx*>(p)->zero_j();
  return ORC_OK;
}
int orc_stage_push_deposit(void* p) { return static_cast<Ctx*>(p)->push_deposit_all(); }

// CIC gather of prognostic component comp (0..2 = d, 3..5 = b) at grid position x3.
int orc_gather(void* p, int comp, const double* x3, double* out) {
  Ctx* ctx = static_cast<Ctx*>(p);
  if (comp < 0 || comp > 5) return ORC_ERR_INVALID;
  return ctx->gather(comp, x3, out) ? ORC_OK : ORC_ERR_CFL;
}

// Field strength B0 of Wald's field for contexts created with ORC_ANALYTIC_WALD.
void orc_set_wald_b0(void* p, double B0) { static_cast<Ctx*>(p)->wald_B0 = B0; }

int orc_accel(void* p, double qm, const double* x4, const double* u4, double* out4) {
  Ctx* ctx = static_cast<Ctx*>(p);
  return ctx->accel(x4, u4, qm, out4) ? ORC_OK : ORC_ERR_CFL;
}

// Deposit one move x1 -> x2 into the context's J (adds to it).
int orc_deposit(void* p, const double* x1, const double* x2, double qmacro, double gbar) {
  Ctx* ctx = static_cast<Ctx*>(p);
  return ctx->deposit(x1, x2, qmacro, gbar, ctx->J) ? ORC_OK : ORC_ERR_CFL;
}

void orc_face_weights(void* p, int K, const double* P, const int* cell, double* W4) {
  static_cast<Ctx*>(p)->face_weights(K, P, cell, W4);
}

// Moves of the last push of a species: n_out in/out, x0/x1 planar (3, n).
int orc_last_moves(void* p, int species, long long* n_inout, double* x0, double* x1, uint32_t* ids) {
  Ctx* ctx = static_cast<Ctx*>(p);
  if (species < 0 || species >= (int)ctx->sp.size()) return ORC_ERR_INVALID;
  const Species& s = ctx->sp[species];
  const long long n = (long long)s.last_id.size();
  if (!x0) {
    *n_inout = n;
    return ORC_OK;
  }
  if (*n_inout < n) return ORC_ERR_INVALID;
  for (int ax = 0; ax < 3; ++ax)
    for (long long i = 0; i < n; ++i) {
      x0[ax * n + i] = s.last_x0[ax][i];
      x1[ax * n + i] = s.last_x1[ax][i];
    }
  for (long long i = 0; i < n; ++i) ids[i] = s.last_id[i];
  *n_inout = n;
  return ORC_OK;
}

// stats: removed_horizon, removed_outer, f_fallbacks, steps
void orc_get_stats(void* p, long long* out4) {
  Ctx* ctx = static_cast<Ctx*>(p);
  out4[0] = ctx->stat_removed_horizon;
  out4[1] = ctx->stat_removed_outer;
  out4[2] = ctx->stat_fallback;
  out4[3] = ctx->stat_steps;
}

// Largest |Christoffel terms of Eq. 11| seen, and the largest sum of the magnitudes of
// their individual products (the scale cancellation has to beat).
void orc_gamma_terms(void* p, double* out2) {
  Ctx* ctx = static_cast<Ctx*>(p);
  out2[0] = ctx->gterm_max;
  out2[1] = ctx->gterm_scale;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
