// Internal types shared by the CUDA translation units of the GRPIC library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace grpic {

constexpr uint32_t kDead = 0xffffffffu;  // sort key of a removed particle
// Transient key of a particle handed to the near-hole pass of the split FP32-mixed push (set
// by the classification, overwritten by the push); cell keys stay below 2^31.
constexpr uint32_t kNear = 0xfffffffeu;

// Device status word (sticky until read by the host).
enum : unsigned {
  ST_NONFINITE = 1u,
  ST_CFL = 2u,
  ST_RANGE = 4u,        // an index had to be clamped (a position left the grid)
  ST_LOAD_INVALID = 8u, // a loaded particle was outside the domain or had no u^4 solution
  ST_LOAD_ERGO = 16u,   // contravariant u^i given where g_44 >= 0
};

struct DevStatus {
  unsigned flags;
  unsigned pad;
  unsigned long long removed_horizon;
  unsigned long long removed_outer;
  unsigned long long fallbacks;
  unsigned long long fp64_evals;
  unsigned long long pushed;  // particle-steps advanced
};

// Geometry and constants of one simulation, passed by value to every kernel.
struct Grid {
  int nx, ny, nz;
  long long ncell;
  double m, a, c, dt;
  double xc, yc, zc;  // centre of mass in grid coordinates
  double r_plus, r_exc;
  double r_fp64;  // FP32-mixed: promote metric evaluations to FP64 where r < r_fp64
  int quad_order;
  unsigned flags;
  // field-step constants, formed once on the host in both precisions: dx^4 = c dt and 4 pi / c
  double dx4, four_pi_c;
  float dx4_f, four_pi_c_f;
  // absorbing layers: inner relaxation k_in from r_exc (falling to 0 at r_abs = r_+), outer k_out over
  // w_out cells; 0 -> no layer
  double k_in, k_out, r_abs;
  int w_out;
  double inv_w;           // 1 / w_out
  float k_out_f, inv_w_f;  // the outer layer's constants in FP32
  // box of cells (origin, extent per axis) holding every location of the inner layer; its table
  // of relaxations is 6 x kboxn[0] x kboxn[1] x kboxn[2] values (location-major)
  int kbox0[3], kboxn[3];
};

template <typename T>
__host__ __device__ inline T grid_dx4(const Grid& g) {
  if constexpr (sizeof(T) == sizeof(float)) return g.dx4_f; else return g.dx4;
}
template <typename T>
__host__ __device__ inline T grid_four_pi_c(const Grid& g) {
  if constexpr (sizeof(T) == sizeof(float)) return g.four_pi_c_f; else return g.four_pi_c;
}

// The field state a kernel reads: the current d and b and the current density J (FP64).
template <typename T>
struct Fields {
  T* d[3];  // contravariant (F^x4, F^y4, F^z4) on edges
  T* b[3];  // covariant (F_yz, F_zx, F_xy) on faces
  double* J[3];
};

// Both buffers of the field ping-pong pairs, the target of the absorbing layers (d planes 0-2, b
// planes 3-5; null without layers) and the per-cell location flags (bit l: location l advanced;
// bit 6: an advanced location of the cell lies in an absorbing layer; bit 7: in the inner one;
// bit 8 + l: location l excised).  The field updates write the other buffer.
constexpr unsigned kLayerBit = 1u << 6;
constexpr unsigned kInnerBit = 1u << 7;
template <typename T>
struct FieldStore {
  T* d[2][3];
  T* b[2][3];
  double* J[3];
  const T* tgt[6];
  const T* kin;  // the inner layer's relaxation table (null without it)
  const uint16_t* loc;
};

// Metric constants of the field kernels in the field type, converted once on the host (this GPU
// converts FP64 to FP32 on its reduced-rate FP64 pipe): centre, spin, 2m, dx^4 and 4 pi / c.
template <typename T>
struct FieldConsts {
  T xc, yc, zc, a, a2, two_m, dx4, four_pi_c;
  bool massive;
};
template <typename T>
__host__ __device__ inline FieldConsts<T> field_consts(const Grid& g) {
  FieldConsts<T> K;
  K.xc = (T)g.xc;
  K.yc = (T)g.yc;
  K.zc = (T)g.zc;
  K.a = (T)g.a;
  K.a2 = K.a * K.a;
  K.two_m = (T)(2.0 * g.m);
  K.dx4 = grid_dx4<T>(g);
  K.four_pi_c = grid_four_pi_c<T>(g);
  K.massive = g.m > 0.0;
  return K;
}

// B half-step: b_out = b_base - coef curl e(b_src, d) at advanced face locations, b_base copied
// elsewhere (not written when inplace: b_out == b_base); relaxed toward tgt in the absorbing
// layers when tgt is set (the second half-step).
template <typename T>
struct BStepArgs {
  const T* src[3];
  const T* base[3];
  T* out[3];
  const T* d[3];
  const T* tgt[3];
  const T* kin;
  const uint16_t* loc;
  FieldConsts<T> K;
  T coef;
  bool inplace;
};

// E step: d_out = d + dx4 (4 pi/c J - div h(b, d*)) at advanced edge locations, d copied
// elsewhere; d* = d + (dx4/2)(4 pi/c J - div h(b, d)) with pred, else d.  Relaxed toward tgt in
// the absorbing layers when tgt is set.
template <typename T>
struct EStepArgs {
  const T* b[3];
  const T* d[3];
  T* out[3];
  const T* tgt[3];
  const T* kin;
  const double* J[3];
  const uint16_t* loc;
  FieldConsts<T> K;
  bool pred;
};

// Patches of a grid for the field launches: ntx x nty patches of (x, y) columns, z in chunks.
struct TileGrid {
  int ntx, nty, ntz, zchunk;
  __host__ __device__ long long count() const { return (long long)ntx * nty * ntz; }
};

template <typename T>
struct Particles {
  T* x[4];  // x^1..x^3 in grid units; x[3] holds x^4 - c t_n
  T* u[4];
  uint32_t* id;
  uint32_t* key;
  long long n;       // entries in the arrays (live + removed-not-yet-sorted)
  const int* n_dev;  // live+flagged count after the last sort (device)
};

__host__ __device__ inline long long cell_index(const Grid& g, int i, int j, int k) {
  return ((long long)k * g.ny + j) * g.nx + i;
}

// ---- launchers (defined in fields.cu, push.cu, sort.cu) --------------------------------
void launch_location_flags(const Grid& g, uint16_t* loc, cudaStream_t st);
// The inner absorbing layer's relaxation over the box g.kbox0 / g.kboxn (6 values per cell).
template <typename T>
void launch_inner_kappa_table(const Grid& g, T* kin, cudaStream_t st);
// B half-steps (Eq. 10) and the E step (Eq. 12); sms sizes the z chunks of the launch.
template <typename T>
void launch_b_step(const Grid& g, const BStepArgs<T>& A, int sms, cudaStream_t st);
template <typename T>
void launch_e_step(const Grid& g, const EStepArgs<T>& A, int sms, cudaStream_t st);
// Patch tables of one instance for the batched field launches.
void batch_field_tiles(const Grid& g, bool fp32, TileGrid* btiles, TileGrid* etiles);
template <typename T>
void launch_uniform_field(const Grid& g, const Fields<T>& F, const double E[3], const double B[3], cudaStream_t st);
template <typename T>
void launch_convert_in(T* dst, const double* src, long long n, cudaStream_t st);
template <typename T>
void launch_convert_out(double* dst, const T* src, long long n, cudaStream_t st);
// The contravariant face components (F^yz, F^zx, F^xy) of every cell as the E step converts them,
// into h3 (3 planes of FP64, device)
template <typename T>
void launch_contra_h(const Grid& g, const Fields<T>& F, const uint16_t* loc, double* h3, cudaStream_t st);
// dst[i] += src[i], FP64
void launch_add_f64(double* dst, const double* src, long long n, cudaStream_t st);

struct Species {
  double qm, qmacro;
};

// Constants of one push launch in the arithmetic type T, built once on the host (for the batch:
// once per instance and species, in its descriptor), plus their FP64 values for the promoted
// evaluations of the FP32-mixed policy.
template <typename T>
struct Consts {
  T xc, yc, zc, m, a;        // centre of mass, mass, spin
  T a2, two_m;               // a^2, 2m
  T c, dt, inv_dt, inv_c, cdt;
  T qm, qmacro;              // q/m (Lorentz term of Eq. 15), macro-particle charge (deposit)
  T rcheck2;                 // removal screen: r^2 below this -> FP64 test against r_+
  float r_fp64, r2_fp64;     // FP32-mixed: promote where the FP32 r is below r_fp64
  bool massive;              // m > 0
  bool gamma_in_j;           // J = rho gamma v (else the plain Umeda flux)
  double dxc, dyc, dzc, dm, da, da2, r_plus;
};

template <typename T>
__host__ __device__ inline Consts<T> make_consts(const Grid& g, const Species& sp) {
  Consts<T> C;
  C.xc = (T)g.xc;
  C.yc = (T)g.yc;
  C.zc = (T)g.zc;
  C.m = (T)g.m;
  C.a = (T)g.a;
  C.a2 = C.a * C.a;
  C.two_m = T(2) * C.m;
  C.c = (T)g.c;
  C.dt = (T)g.dt;
  C.inv_dt = T(1) / (T)g.dt;
  C.inv_c = T(1) / (T)g.c;
  C.cdt = (T)(g.c * g.dt);
  C.qm = (T)sp.qm;
  C.qmacro = (T)sp.qmacro;
  C.rcheck2 = (T)(1.2 * g.r_plus * g.r_plus + 1.0);
  C.r_fp64 = (float)g.r_fp64;
  C.r2_fp64 = C.r_fp64 > 0.f ? C.r_fp64 * C.r_fp64 : -1.f;  // negative: never promote
  C.massive = g.m > 0.0;
  C.gamma_in_j = (g.flags & 1u) == 0;
  C.dxc = g.xc;
  C.dyc = g.yc;
  C.dzc = g.zc;
  C.dm = g.m;
  C.da = g.a;
  C.da2 = g.a * g.a;
  C.r_plus = g.r_plus;
  return C;
}

template <typename T>
void launch_push_deposit(const Grid& g, const Fields<T>& F, const Particles<T>& P, const Species& sp,
                         DevStatus* st, bool mixed, double t_offset, cudaStream_t stream);

// Far-field criterion of the FP32-mixed push: every RK4 stage and quadrature node of a
// particle-step lies within 2 sqrt(3) < 4 cells of x_n (stages move less than a cell; nodes lie
// in the cells of x_n and x_{n+1}, neighbours since |dx^i| < 1), and r >= R - |a| (Eq. 6), so a
// particle with R(x_n) >= r_fp64 + |a| + 4 never needs the FP64 policy and every node of its
// deposit has R > |a|.
__host__ __device__ inline double near_radius(const Grid& g) {
  return (g.r_fp64 > 0.0 ? g.r_fp64 : 0.0) + (g.a < 0.0 ? -g.a : g.a) + 4.0;
}

// Far-field deposit from per-cell polynomial fits of the Eq. 18 integrand (area_table.cu):
// kAreaTableStride float4 (256 bytes, two cache lines) per cell, indexed by the cell's linear index.
// The fit of face orientation K (kFitTerms coefficients; term t enumerates u^i v^j w^k for j = 0..4,
// i = 0..4-j, k = 0..4-i-j) takes the 5 float4 from 5K: four FP32 (terms 0, 1, 5, 15: the constant and
// the linear terms w, u, v), then the other 31 terms in FP16 in term order and one zero; float4 15 is
// zero.  The FP16 terms (second order and up: ~m / r^3 and smaller) keep absolute errors below 2e-7.
// table_radius: a warp takes the fits only if every particle has R(x_n) >= table_radius
// (>= near_radius; where the fit's truncation error, ~m / r^6, leaves the weights within a few 1e-9
// of Q = 2 Gauss quadrature).
constexpr int kAreaTableStride = 16;
constexpr int kFitTerms = 35;
__host__ __device__ constexpr bool fit_term_fp32(int t) { return t == 0 || t == 1 || t == 5 || t == 15; }
double table_radius(const Grid& g);
void launch_area_table(const Grid& g, float4* tab, cudaStream_t st);

// Split FP32-mixed push.  near_radius: particles with R(x_n) below it are classified near
// (marked kNear, listed; count[0] = list length, count[1] = work cursor) and pushed by
// launch_push_near (nblocks persistent blocks; new sort keys to keys[slot]); the rest by launch_push_far (FP32 only; minb selects
// the register budget), concurrently.  launch_near_keys then copies keys[slot] to P.key.
void launch_classify_near(const Grid& g, const Particles<float>& P, uint32_t* list, int* count,
                          cudaStream_t stream);
void launch_push_far(const Grid& g, const Fields<float>& F, const Particles<float>& P, const Species& sp,
                     DevStatus* st, int minb, cudaStream_t stream);
void launch_push_near(const Grid& g, const Fields<float>& F, const Particles<float>& P, const Species& sp,
                      DevStatus* st, const uint32_t* list, uint32_t* keys, int* count, int nblocks,
                      cudaStream_t stream);
void launch_near_keys(const Particles<float>& P, const uint32_t* list, const uint32_t* keys, const int* count,
                      int nblocks, cudaStream_t stream);
// A multiplier coprime to n near 0.618 n: blockIdx * m mod n permutes n work items evenly.
unsigned coprime_multiplier(unsigned n);

// Block -> work-chunk map of the push launches: groups of 2^lg consecutive chunks are permuted,
// group g -> g * perm mod (number of full groups), perm coprime to that number (1 keeps the order;
// a partial last group stays in place).  Cell-sorted particles put the FP64-heavy chunks near the
// hole in one contiguous run; the permutation spreads them over the whole launch, so the FP64
// pipes of all SMs share that work alongside FP32 work, while the blocks of a group, which run at
// about the same time, keep neighbouring cells together (their field stencils and J nodes stay in
// L2).  Larger groups favour that locality, smaller ones the spreading of FP64 work.
__device__ __forceinline__ unsigned spread_chunk(unsigned b, unsigned n, unsigned perm, int lg) {
  const unsigned nfull = n >> lg;
  if (perm == 1u || b >= (nfull << lg)) return b;
  const unsigned mask = (1u << lg) - 1u;
  return ((unsigned)(((unsigned long long)(b >> lg) * perm) % nfull) << lg) | (b & mask);
}
inline unsigned spread_multiplier(unsigned n, int lg) { return coprime_multiplier(n >> lg); }
// group size of the batched push
constexpr int kBatchSpreadLog2 = 4;
// log2 of a push spread group size (tuning value: 1, 2, 4, ... 64)
inline int spread_log2(int group) {
  int lg = 0;
  while ((1 << lg) < group) ++lg;
  return lg;
}
// Unsplit alternative: one launch, far-field or FP32-mixed code chosen per warp by the same
// near_radius criterion.  atab (non-null, Q = 2, no tile): far-field warps deposit with the
// per-cell area fits, and the criterion becomes table_radius.
void launch_push_select(const Grid& g, const Fields<float>& F, const Particles<float>& P, const Species& sp,
                        DevStatus* st, int minb, bool tile, int spread, const float4* atab, cudaStream_t stream);

template <typename T>
void launch_load_particles(const Grid& g, const Particles<T>& P, long long n, const double* x4, const double* u4,
                           const uint32_t* ids, int umode, double ct_now, DevStatus* st, cudaStream_t stream);
template <typename T>
void launch_unload_particles(const Particles<T>& P, long long n, double* x4, double* u4, uint32_t* ids,
                             double ct_now, cudaStream_t stream);

// Diagnostics (diag.cu): CIC charge density (times gamma with with_gamma) added into rho, and
// the Gauss residual div E - 4 pi rho with the max |residual| over nodes [lo, n-1-lo]^3.
template <typename T>
void launch_charge_density(const Particles<T>& P, double q, const Grid& g, bool with_gamma, double* rho,
                           cudaStream_t stream);
template <typename T>
void launch_gauss(const Fields<T>& F, const double* rho, const Grid& g, int lo, double* res,
                  unsigned long long* maxabs, cudaStream_t stream);
// Invariant statistics (diag.cu): mode 0 records the tracked particles' E and L, mode 1 compares;
// acc: invariant_acc_bytes() of zeroed device memory accumulating over the species launched.
template <typename T>
void launch_invariants(const Grid& g, const Particles<T>& P, int mode, int stride, double* e0, double* l0,
                       long long nslots, void* acc, cudaStream_t stream);
template <typename T>
void launch_max_id(const Particles<T>& P, unsigned long long* max_id, cudaStream_t stream);
size_t invariant_acc_bytes();
constexpr int kInvariantStride = 64;  // tracked subsample: ids divisible by this

// Counting sort by cell of one species; removed particles (key == kDead) are dropped.
// counts: nbins+1 ints, offsets: nbins+1 ints, blocks: scan scratch; n_out: device int.
struct SortScratch {
  int* counts;
  int* offsets;
  int* blocks;
  int nblocks;
};
template <typename T>
void launch_sort(const Grid& g, const Particles<T>& src, const Particles<T>& dst, const SortScratch& s,
                 int* n_out, cudaStream_t stream);

// ---- batched engine -------------------------------------------------------------------------
// Every stage of a batched step is one launch over a device table of work blocks; each block
// belongs to exactly one instance (work is padded to whole blocks), so per-instance state and
// warp-level reductions stay block-uniform.  Kernels loop over the table grid-stride.
struct BlockEntry {
  int inst;   // instance (field stages) or instance * 4 + species (particle stages)
  int block;  // block index within that instance's work
};

template <typename T>
struct SpeciesDesc {
  Consts<T> C;          // launch constants of this (instance, species)
  float r_near2;        // near_radius^2 of the instance (FP32-mixed far-field criterion)
  double qm, qmacro;
  Particles<T> buf[2];  // the two ping-pong buffers (n = work upper bound, n_dev = live count)
  int* cur;             // device int: index of the current buffer
  long long bin_base;   // first sort bin of this (instance, species) in the batch's bin array
  int active;
};

template <typename T>
struct InstDesc {
  Grid g;
  FieldConsts<float> K32;  // field-kernel constants in both types (the batch is FP32 or FP64)
  FieldConsts<double> K64;
  FieldStore<T> FS;  // b[0]: b at the start of a step (b^{n-1/2}), b[1]: b^n
  int* dcur;         // device: which d buffer holds the current d
  TileGrid btiles, etiles;
  DevStatus* st;
  SpeciesDesc<T> sp[4];
};

template <typename T>
struct BatchTables {
  const InstDesc<T>* desc;
  const BlockEntry* btile;  // B-step patches of every instance
  int nbtile;
  const BlockEntry* etile;  // E-step patches
  int netile;
  const BlockEntry* all;   // all cells, 256 per block
  int nall;
  const BlockEntry* part;  // particles of (instance, species), 128 per block
  int npart;
  int* counts;             // sort bins of every (instance, species)
  int* offsets;
  int* tiles;
  long long nbins;
  const int* pairs;        // instance * 4 + species of every loaded species
  int npairs;
  int* pair_base;          // exclusive prefix at each pair's first bin (per step)
  int persist_blocks;      // grid size of the persistent launches
  int persist_field_blocks;  // grid size of the persistent field launches (512-thread blocks)
};

template <typename T>
void launch_batch_b_half(const BatchTables<T>& bt, int which, bool literal, cudaStream_t st);
template <typename T>
void launch_batch_e_step(const BatchTables<T>& bt, bool literal, cudaStream_t st);
template <typename T>
void launch_batch_zero_j(const BatchTables<T>& bt, cudaStream_t st);
// flip every instance's d parity (end of a batched step)
template <typename T>
void launch_batch_flip_d(const BatchTables<T>& bt, int ninst, cudaStream_t st);
template <typename T>
void launch_batch_push(const BatchTables<T>& bt, int quad_order, cudaStream_t st);
template <typename T>
void launch_batch_sort(const BatchTables<T>& bt, cudaStream_t st);

}  // namespace grpic
