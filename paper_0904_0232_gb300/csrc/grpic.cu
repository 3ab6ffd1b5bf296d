// Host side of the GRPIC C ABI (include/grpic.h): context lifecycle, memory, the
// stream-ordered timestep pipeline of Sec. 2.2 (Fig. 1) and the device status word.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/grpic.h"
#include "common.cuh"

using namespace grpic;

namespace grpic {
int scan_tiles(long long nbins);
}

namespace {

constexpr int kMaxSpecies = 4;

struct SpeciesStore {
  double qm = 0.0, qmacro = 0.0;
  long long n = 0;    // array entries (upper bound of the live count)
  long long cap = 0;  // capacity in particles
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  int* n_dev = nullptr;
  int* n_shadow = nullptr;  // pinned host copy of n_dev
  int* near_n = nullptr;    // split push: near-hole list length and work cursor (2 device ints)
  cudaEvent_t shadow_ev = nullptr;
  bool shadow_pending = false;
  bool loaded = false;
};

}  // namespace

struct grpic_ctx {
  grpic_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  Grid g{};
  bool mixed = false;
  size_t tsize = 8;
  std::string err;
  // split FP32-mixed push: second stream (higher priority) and its fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int sms = 0;
  grpic_tuning tune{4, 4, 1, 1, 0, 0, 1, 0};
  void* fields = nullptr;  // 12 planes of T: d buffers 0 and 1 (3 planes each), b buffers 0 and 1
  void* tgt = nullptr;     // absorbing layers: 6 planes of T, the target d and b (null without layers)
  void* kin = nullptr;     // inner absorbing layer: relaxation table over g.kbox0 / g.kboxn (T)
  double* J = nullptr;     // 3 planes
  float4* atab = nullptr;  // per-cell area fits of the far-field deposit (built when tune.area_table is set)
  uint16_t* loc = nullptr;  // per-cell location flags
  // field ping-pong state: buffer of the current d and b; bprev: buffer holding b^{n-1/2} after the
  // first B half-step (time-centred second half-step)
  int dcur = 0, bcur = 0, bprev = 0;
  DevStatus* st = nullptr;
  DevStatus* st_host = nullptr;  // pinned
  SortScratch sort{};
  SpeciesStore sp[kMaxSpecies];
  long long steps = 0;
  long long pushes = 0;
  grpic_status step_status = GRPIC_OK;  // status of this context after the last batched step  // push stages run: particle x^4 is stored relative to c dt * pushes
  int since_sort = 0;
  grpic_stats totals{};
  // invariant baselines: per species E and L of the tracked particles, by id / stride
  double* inv_e0[kMaxSpecies] = {nullptr, nullptr, nullptr, nullptr};
  double* inv_l0[kMaxSpecies] = {nullptr, nullptr, nullptr, nullptr};
  long long inv_slots[kMaxSpecies] = {0, 0, 0, 0};
  // tracing
  long long launches = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending {
    cudaEvent_t a, b;
    int stage;
  };
  std::vector<Pending> pending;
  double prof_ms[6] = {0, 0, 0, 0, 0, 0};
  long long prof_cnt[6] = {0, 0, 0, 0, 0, 0};
};

namespace {

void* dev_alloc(grpic_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (c->cfg.alloc) return c->cfg.alloc(bytes, c->cfg.alloc_user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(grpic_ctx* c, void* p) {
  if (!p) return;
  if (c->cfg.free_fn) {
    c->cfg.free_fn(p, c->cfg.alloc_user);
    return;
  }
  cudaFree(p);
}

grpic_status fail(grpic_ctx* c, grpic_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

grpic_status cuda_check(grpic_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return GRPIC_OK;
  return fail(c, GRPIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t particle_bytes(const grpic_ctx* c) { return 8 * c->tsize + 2 * sizeof(uint32_t); }

template <typename T>
T* field_plane(grpic_ctx* c, bool is_b, int buf, int q) {
  return static_cast<T*>(c->fields) + (size_t)((is_b ? 6 : 0) + 3 * buf + q) * c->g.ncell;
}

// Plane q of the absorbing layers' target (0-2: d, 3-5: b), or null without layers.
template <typename T>
T* target_plane(grpic_ctx* c, int q) {
  return c->tgt ? static_cast<T*>(c->tgt) + (size_t)q * c->g.ncell : nullptr;
}

// The current d and b become the absorbing layers' target.
void snapshot_target(grpic_ctx* c) {
  if (!c->tgt) return;
  const size_t bytes = 3 * (size_t)c->g.ncell * c->tsize;
  char* t = static_cast<char*>(c->tgt);
  const char* f = static_cast<const char*>(c->fields);
  cudaMemcpyAsync(t, f + (size_t)c->dcur * bytes, bytes, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(t + bytes, f + (size_t)(2 + c->bcur) * bytes, bytes, cudaMemcpyDeviceToDevice, c->stream);
}

// The current field state (what the push, the diagnostics and get/set_fields see).
template <typename T>
Fields<T> fields_view(grpic_ctx* c) {
  Fields<T> F;
  for (int q = 0; q < 3; ++q) {
    F.d[q] = field_plane<T>(c, false, c->dcur, q);
    F.b[q] = field_plane<T>(c, true, c->bcur, q);
    F.J[q] = c->J + (size_t)q * c->g.ncell;
  }
  return F;
}

template <typename T>
Particles<T> particles_view(grpic_ctx* c, int s, int which) {
  SpeciesStore& S = c->sp[s];
  Particles<T> P;
  char* base = static_cast<char*>(S.buf[which]);
  const size_t cap = (size_t)S.cap;
  for (int q = 0; q < 4; ++q) {
    P.x[q] = reinterpret_cast<T*>(base + q * cap * sizeof(T));
    P.u[q] = reinterpret_cast<T*>(base + (4 + q) * cap * sizeof(T));
  }
  P.id = reinterpret_cast<uint32_t*>(base + 8 * cap * sizeof(T));
  P.key = reinterpret_cast<uint32_t*>(base + 8 * cap * sizeof(T) + cap * sizeof(uint32_t));
  P.n = S.n;
  P.n_dev = S.n_dev;
  return P;
}

// Refresh the host upper bound of the live count from the last completed shadow copy.
void refresh_count(SpeciesStore& S) {
  if (S.shadow_pending && cudaEventQuery(S.shadow_ev) == cudaSuccess) {
    S.n = std::min<long long>(S.n, *S.n_shadow);
    S.shadow_pending = false;
  }
}

bool literal_fields(const grpic_ctx* c) { return (c->cfg.flags & GRPIC_LITERAL_HALF_STEPS) != 0; }

bool split_push(const grpic_ctx* c) {
  return c->mixed && c->g.r_fp64 > 0.0 && !(c->cfg.flags & GRPIC_SINGLE_PUSH_KERNEL);
}

// rho (FP64, nodes) of every loaded species into device memory `rho` (zeroed first).
template <typename T>
void enqueue_rho(grpic_ctx* c, bool with_gamma, double* rho) {
  cudaMemsetAsync(rho, 0, sizeof(double) * (size_t)c->g.ncell, c->stream);
  for (int s = 0; s < kMaxSpecies; ++s) {
    SpeciesStore& S = c->sp[s];
    if (!S.loaded || S.n == 0) continue;
    launch_charge_density<T>(particles_view<T>(c, s, S.cur), S.qmacro, c->g, with_gamma, rho, c->stream);
  }
}

// The area fits the per-warp select push uses, or null.
const float4* area_table_of(const grpic_ctx* c) { return c->tune.area_table ? c->atab : nullptr; }

// Unsplit FP32-mixed push: one launch per species, far-field or mixed code chosen per warp.
void enqueue_select_push(grpic_ctx* c) {
  Fields<float> F = fields_view<float>(c);
  for (int s = 0; s < kMaxSpecies; ++s) {
    SpeciesStore& S = c->sp[s];
    if (!S.loaded || S.n == 0) continue;
    refresh_count(S);
    launch_push_select(c->g, F, particles_view<float>(c, s, S.cur), Species{S.qm, S.qmacro}, c->st,
                       c->tune.far_min_blocks, c->tune.j_tile != 0, c->tune.spread, area_table_of(c), c->stream);
    c->launches += 1;
  }
}

void enqueue_far(grpic_ctx* c, const Fields<float>& F) {
  for (int s = 0; s < kMaxSpecies; ++s) {
    SpeciesStore& S = c->sp[s];
    if (!S.loaded || S.n == 0) continue;
    launch_push_far(c->g, F, particles_view<float>(c, s, S.cur), Species{S.qm, S.qmacro}, c->st,
                    c->tune.far_min_blocks, c->stream);
    c->launches += 1;
  }
}

// Split FP32-mixed push: classify every species on the context stream, then the near-hole
// kernels on the side stream and the far kernels on the context stream, joined at the end, and
// the near particles' sort keys copied into place (with tune.overlap = 0: far kernels, then
// near kernels, all on the context stream).  The near list and the near kernel's keys
// live in the key and id planes of the idle ping-pong buffer (written again only by the next
// sort, which follows the push).
void enqueue_split_push(grpic_ctx* c) {
  Fields<float> F = fields_view<float>(c);
  bool any = false;
  for (int s = 0; s < kMaxSpecies; ++s) {
    SpeciesStore& S = c->sp[s];
    if (!S.loaded || S.n == 0) continue;
    refresh_count(S);
    cudaMemsetAsync(S.near_n, 0, 2 * sizeof(int), c->stream);
    launch_classify_near(c->g, particles_view<float>(c, s, S.cur), particles_view<float>(c, s, 1 - S.cur).key,
                         S.near_n, c->stream);
    c->launches += 1;
    any = true;
  }
  if (!any) return;
  const bool overlap = c->tune.overlap != 0;
  cudaStream_t near_stream = overlap ? c->side : c->stream;
  if (overlap) {
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  } else {
    enqueue_far(c, F);
  }
  const int nb = c->sms * c->tune.near_blocks_per_sm;
  for (int s = 0; s < kMaxSpecies; ++s) {
    SpeciesStore& S = c->sp[s];
    if (!S.loaded || S.n == 0) continue;
    const Particles<float> idle = particles_view<float>(c, s, 1 - S.cur);
    launch_push_near(c->g, F, particles_view<float>(c, s, S.cur), Species{S.qm, S.qmacro}, c->st, idle.key,
                     idle.id, S.near_n, nb, near_stream);
    c->launches += 1;
  }
  if (overlap) {
    enqueue_far(c, F);
    cudaEventRecord(c->ev_join, c->side);
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);
  }
  for (int s = 0; s < kMaxSpecies; ++s) {
    SpeciesStore& S = c->sp[s];
    if (!S.loaded || S.n == 0) continue;
    const Particles<float> idle = particles_view<float>(c, s, 1 - S.cur);
    launch_near_keys(particles_view<float>(c, s, S.cur), idle.key, idle.id, S.near_n, c->sms * 2, c->stream);
    c->launches += 1;
  }
}

template <typename T>
void enqueue_stage(grpic_ctx* c, int stage) {
  Fields<T> F = fields_view<T>(c);
  switch (stage) {
    case GRPIC_STAGE_B_HALF:
    case GRPIC_STAGE_B_HALF2: {
      // first half: b_cur -> the other buffer (b_cur kept as b^{n-1/2}); second half, time-centred:
      // b^{n+1/2} = b^{n-1/2} - dx4 curl e(b^n, d) over the saved buffer; literal: b -= dx4/2 curl e
      // into the other buffer
      const bool second = stage == GRPIC_STAGE_B_HALF2;
      const bool centred = second && !literal_fields(c);
      const int out = centred ? c->bprev : 1 - c->bcur;
      BStepArgs<T> A;
      for (int q = 0; q < 3; ++q) {
        A.src[q] = field_plane<T>(c, true, c->bcur, q);
        A.base[q] = field_plane<T>(c, true, centred ? c->bprev : c->bcur, q);
        A.out[q] = field_plane<T>(c, true, out, q);
        A.d[q] = F.d[q];
        A.tgt[q] = second ? target_plane<T>(c, 3 + q) : nullptr;
      }
      A.kin = static_cast<const T*>(c->kin);
      A.loc = c->loc;
      A.K = field_consts<T>(c->g);
      const T dx4 = grid_dx4<T>(c->g);
      A.coef = centred ? dx4 : dx4 * T(0.5);
      A.inplace = centred;
      launch_b_step<T>(c->g, A, c->sms, c->stream);
      c->launches += 1;
      if (!second) c->bprev = c->bcur;
      c->bcur = out;
      break;
    }
    case GRPIC_STAGE_ZERO_J:
      cudaMemsetAsync(c->J, 0, sizeof(double) * 3 * (size_t)c->g.ncell, c->stream);
      break;
    case GRPIC_STAGE_PUSH_DEPOSIT:
      if (split_push(c)) {
        if (c->tune.split)
          enqueue_split_push(c);
        else
          enqueue_select_push(c);
      } else {
        for (int s = 0; s < kMaxSpecies; ++s) {
          SpeciesStore& S = c->sp[s];
          if (!S.loaded || S.n == 0) continue;
          refresh_count(S);
          Species spc{S.qm, S.qmacro};
          launch_push_deposit<T>(c->g, F, particles_view<T>(c, s, S.cur), spc, c->st, c->mixed, 0.0, c->stream);
          c->launches += 1;
        }
      }
      c->pushes += 1;
      break;
    case GRPIC_STAGE_E: {
      EStepArgs<T> A;
      for (int q = 0; q < 3; ++q) {
        A.b[q] = F.b[q];
        A.d[q] = F.d[q];
        A.out[q] = field_plane<T>(c, false, 1 - c->dcur, q);
        A.J[q] = F.J[q];
        A.tgt[q] = target_plane<T>(c, q);
      }
      A.kin = static_cast<const T*>(c->kin);
      A.loc = c->loc;
      A.K = field_consts<T>(c->g);
      A.pred = !literal_fields(c);
      launch_e_step<T>(c->g, A, c->sms, c->stream);
      c->launches += 1;
      c->dcur = 1 - c->dcur;
      break;
    }
    case GRPIC_STAGE_SORT:
      for (int s = 0; s < kMaxSpecies; ++s) {
        SpeciesStore& S = c->sp[s];
        if (!S.loaded) continue;
        launch_sort<T>(c->g, particles_view<T>(c, s, S.cur), particles_view<T>(c, s, 1 - S.cur), c->sort, S.n_dev,
                       c->stream);
        c->launches += S.n > 0 ? 6 : 4;
        S.cur = 1 - S.cur;
        cudaMemcpyAsync(S.n_shadow, S.n_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        cudaEventRecord(S.shadow_ev, c->stream);
        S.shadow_pending = true;
      }
      break;
    default:
      break;
  }
}

cudaEvent_t pool_event(grpic_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Fold finished stage timings into the totals (called after the stream is synchronised).
void collect_profile(grpic_ctx* c) {
  for (const auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.stage] += ms;
      c->prof_cnt[p.stage] += 1;
    }
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
  cudaGetLastError();
}

void enqueue_stage_any(grpic_ctx* c, int stage) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->profiling) {
    a = pool_event(c);
    b = pool_event(c);
    cudaEventRecord(a, c->stream);
  }
  if (c->mixed)
    enqueue_stage<float>(c, stage);
  else
    enqueue_stage<double>(c, stage);
  if (c->profiling) {
    cudaEventRecord(b, c->stream);
    c->pending.push_back({a, b, stage});
  }
}

// One timestep (Sec. 2.2): B half, J = 0, push + deposit, B half, E; then removal + sort.
void enqueue_step(grpic_ctx* c) {
  enqueue_stage_any(c, GRPIC_STAGE_B_HALF);
  enqueue_stage_any(c, GRPIC_STAGE_ZERO_J);
  enqueue_stage_any(c, GRPIC_STAGE_PUSH_DEPOSIT);
  enqueue_stage_any(c, GRPIC_STAGE_B_HALF2);
  enqueue_stage_any(c, GRPIC_STAGE_E);
  c->steps += 1;
  if (++c->since_sort >= std::max(1, c->tune.sort_interval)) {
    enqueue_stage_any(c, GRPIC_STAGE_SORT);
    c->since_sort = 0;
  }
}

grpic_status read_status(grpic_ctx* c) {
  grpic_status s = cuda_check(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                                                 c->stream),
                              "status copy");
  if (s != GRPIC_OK) return s;
  s = cuda_check(c, cudaStreamSynchronize(c->stream), "stream synchronize");
  if (s != GRPIC_OK) return s;
  collect_profile(c);
  const DevStatus h = *c->st_host;
  c->totals.removed_horizon = (int64_t)h.removed_horizon;
  c->totals.removed_outer = (int64_t)h.removed_outer;
  c->totals.gamma_fallbacks = (int64_t)h.fallbacks;
  c->totals.fp64_evals = (int64_t)h.fp64_evals;
  c->totals.particle_steps = (int64_t)h.pushed;
  if (h.flags) {
    // clear the sticky flags now that they are reported
    cudaMemsetAsync(&c->st->flags, 0, sizeof(unsigned), c->stream);
    cudaStreamSynchronize(c->stream);
    if (h.flags & ST_NONFINITE) return fail(c, GRPIC_ERR_NONFINITE, "non-finite particle state");
    if (h.flags & (ST_CFL | ST_RANGE))
      return fail(c, GRPIC_ERR_CFL, "a particle moved a cell or more in one step (or left the grid)");
    if (h.flags & ST_LOAD_ERGO)
      return fail(c, GRPIC_ERR_INVALID, "contravariant u^i given where g_44 >= 0 (ergoregion): ambiguous u^4");
    if (h.flags & ST_LOAD_INVALID)
      return fail(c, GRPIC_ERR_INVALID, "particle outside [1, n-2] or without a future-directed unit u");
  }
  return GRPIC_OK;
}

grpic_status ensure_capacity(grpic_ctx* c, int s, long long n) {
  SpeciesStore& S = c->sp[s];
  long long want = std::max<long long>(n, c->cfg.max_particles);
  if (c->cfg.max_particles > 0 && n > c->cfg.max_particles)
    return fail(c, GRPIC_ERR_CAPACITY, "more particles than max_particles");
  if (S.cap >= want && S.buf[0]) return GRPIC_OK;
  for (int b = 0; b < 2; ++b) {
    dev_free(c, S.buf[b]);
    S.buf[b] = nullptr;
  }
  const size_t bytes = (size_t)std::max<long long>(want, 1) * particle_bytes(c);
  for (int b = 0; b < 2; ++b) {
    S.buf[b] = dev_alloc(c, bytes);
    if (!S.buf[b]) return fail(c, GRPIC_ERR_OOM, "particle store allocation failed");
  }
  S.cap = std::max<long long>(want, 1);
  return GRPIC_OK;
}

}  // namespace

extern "C" {

const char* grpic_status_string(grpic_status s) {
  switch (s) {
    case GRPIC_OK: return "GRPIC_OK";
    case GRPIC_ERR_INVALID: return "GRPIC_ERR_INVALID";
    case GRPIC_ERR_OOM: return "GRPIC_ERR_OOM";
    case GRPIC_ERR_CUDA: return "GRPIC_ERR_CUDA";
    case GRPIC_ERR_CFL: return "GRPIC_ERR_CFL";
    case GRPIC_ERR_NONFINITE: return "GRPIC_ERR_NONFINITE";
    case GRPIC_ERR_TIMEOUT: return "GRPIC_ERR_TIMEOUT";
    case GRPIC_ERR_AGAIN: return "GRPIC_ERR_AGAIN";
    case GRPIC_ERR_CAPACITY: return "GRPIC_ERR_CAPACITY";
    case GRPIC_ERR_UNSTABLE: return "GRPIC_ERR_UNSTABLE";
  }
  return "GRPIC_ERR_UNKNOWN";
}

const char* grpic_last_error(const grpic_ctx* c) { return c ? c->err.c_str() : "null context"; }

grpic_status grpic_create(const grpic_config* cfg, void* stream, grpic_ctx** out) {
  if (!cfg || !out) return GRPIC_ERR_INVALID;
  *out = nullptr;
  if (cfg->nx < 8 || cfg->ny < 8 || cfg->nz < 8) return GRPIC_ERR_INVALID;
  if (!(cfg->m >= 0.0) || !(std::fabs(cfg->a) <= cfg->m) || !(cfg->c > 0.0) || !(cfg->dt > 0.0))
    return GRPIC_ERR_INVALID;
  if (cfg->precision != GRPIC_FP64 && cfg->precision != GRPIC_FP32_MIXED) return GRPIC_ERR_INVALID;
  if (cfg->quad_order < 0 || cfg->quad_order > 3) return GRPIC_ERR_INVALID;
  if ((cfg->alloc == nullptr) != (cfg->free_fn == nullptr)) return GRPIC_ERR_INVALID;
  const long long ncell = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (ncell + 1 >= (1ll << 31)) return GRPIC_ERR_INVALID;
  // Courant condition of the Yee update (Sec. 5): c dt < dx / sqrt(3)
  if (!(cfg->c * cfg->dt < 1.0 / std::sqrt(3.0))) return GRPIC_ERR_CFL;
  if (!(cfg->absorb_inner >= 0.0 && cfg->absorb_inner <= 1.0 && cfg->absorb_outer >= 0.0 &&
        cfg->absorb_outer <= 1.0))
    return GRPIC_ERR_INVALID;
  // one z-slab of a larger run: inside the run's planes; the outer layer's faces would not be its own
  const int nz_total = cfg->nz_total > 0 ? cfg->nz_total : cfg->nz;
  const bool slab = cfg->z_origin != 0 || nz_total != cfg->nz;
  if (cfg->z_origin < 0 || cfg->z_origin + cfg->nz > nz_total || (slab && cfg->absorb_outer > 0.0))
    return GRPIC_ERR_INVALID;

  grpic_ctx* c = new grpic_ctx();
  c->cfg = *cfg;
  if (c->cfg.quad_order == 0) c->cfg.quad_order = 2;
  if (c->cfg.sort_interval <= 0) c->cfg.sort_interval = 1;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&c->device);
  c->mixed = cfg->precision == GRPIC_FP32_MIXED;
  c->tsize = c->mixed ? sizeof(float) : sizeof(double);
  Grid& g = c->g;
  g.nx = cfg->nx;
  g.ny = cfg->ny;
  g.nz = cfg->nz;
  g.ncell = ncell;
  g.m = cfg->m;
  g.a = cfg->a;
  g.c = cfg->c;
  g.dt = cfg->dt;
  g.xc = 0.5 * (cfg->nx - 1);
  g.yc = 0.5 * (cfg->ny - 1);
  g.zc = 0.5 * (nz_total - 1) - cfg->z_origin;
  g.r_plus = cfg->m + std::sqrt(std::max(0.0, cfg->m * cfg->m - cfg->a * cfg->a));
  g.r_exc = cfg->r_excise > 0.0 ? cfg->r_excise : (cfg->absorb_inner > 0.0 ? 0.5 : 1.0) * g.r_plus;
  g.k_in = cfg->absorb_inner;
  g.k_out = cfg->absorb_outer;
  g.r_abs = g.r_plus;
  g.w_out = cfg->absorb_width > 0 ? cfg->absorb_width : 8;
  g.inv_w = 1.0 / g.w_out;
  g.k_out_f = (float)g.k_out;
  g.inv_w_f = (float)g.inv_w;
  // box of cells around the hole holding every location with r < r_+: there r^2 >= R^2 - a^2, so
  // R < sqrt(r_+^2 + a^2), and a location lies within half a cell of its cell's corner
  long long kin_cells = 0;
  for (int ax = 0; ax < 3; ++ax) g.kbox0[ax] = g.kboxn[ax] = 0;
  if (g.k_in > 0.0 && g.m > 0.0) {
    const double hw = std::sqrt(g.r_abs * g.r_abs + g.a * g.a) + 1.0;
    const int n3[3] = {g.nx, g.ny, g.nz};
    const double cen[3] = {g.xc, g.yc, g.zc};
    kin_cells = 1;
    for (int ax = 0; ax < 3; ++ax) {
      const int lo = std::max(2, (int)std::floor(cen[ax] - hw));
      const int hi = std::min(n3[ax] - 3, (int)std::ceil(cen[ax] + hw));
      g.kbox0[ax] = lo;
      g.kboxn[ax] = std::max(0, hi - lo + 1);
      kin_cells *= g.kboxn[ax];
    }
  }
  g.quad_order = c->cfg.quad_order;
  g.flags = cfg->flags;
  g.r_fp64 = (cfg->fp64_radius == 0.0 ? 4.0 : cfg->fp64_radius) * cfg->m;
  if (cfg->fp64_radius < 0.0) g.r_fp64 = -1.0;
  g.dx4 = cfg->c * cfg->dt;
  g.four_pi_c = 4.0 * M_PI / cfg->c;
  g.dx4_f = (float)g.dx4;
  g.four_pi_c_f = (float)g.four_pi_c;

  c->fields = dev_alloc(c, 12 * (size_t)ncell * c->tsize);
  const bool layers = g.k_in > 0.0 || g.k_out > 0.0;
  if (layers) c->tgt = dev_alloc(c, 6 * (size_t)ncell * c->tsize);
  if (kin_cells > 0) c->kin = dev_alloc(c, 6 * (size_t)kin_cells * c->tsize);
  c->J = static_cast<double*>(dev_alloc(c, 3 * (size_t)ncell * sizeof(double)));
  c->loc = static_cast<uint16_t*>(dev_alloc(c, sizeof(uint16_t) * (size_t)ncell));
  c->st = static_cast<DevStatus*>(dev_alloc(c, sizeof(DevStatus)));
  const long long nbins = ncell + 1;
  c->sort.nblocks = scan_tiles(nbins);
  c->sort.counts = static_cast<int*>(dev_alloc(c, sizeof(int) * nbins));
  c->sort.offsets = static_cast<int*>(dev_alloc(c, sizeof(int) * nbins));
  c->sort.blocks = static_cast<int*>(dev_alloc(c, sizeof(int) * (c->sort.nblocks + 1)));
  bool ok = c->fields && c->J && c->loc && c->st && c->sort.counts && c->sort.offsets && c->sort.blocks &&
            (c->tgt || !layers) && (c->kin || kin_cells == 0);
  for (int s = 0; s < kMaxSpecies && ok; ++s) {
    c->sp[s].n_dev = static_cast<int*>(dev_alloc(c, sizeof(int)));
    c->sp[s].near_n = static_cast<int*>(dev_alloc(c, 2 * sizeof(int)));
    ok = c->sp[s].n_dev != nullptr && c->sp[s].near_n != nullptr;
    if (ok) ok = cudaMallocHost(&c->sp[s].n_shadow, sizeof(int)) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&c->sp[s].shadow_ev, cudaEventDisableTiming) == cudaSuccess;
  }
  if (ok) ok = cudaMallocHost(&c->st_host, sizeof(DevStatus)) == cudaSuccess;
  if (ok) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    ok = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess &&
         cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess;
  }
  c->tune.sort_interval = c->cfg.sort_interval;
  if (!ok) {
    grpic_destroy(c);
    return GRPIC_ERR_OOM;
  }
  cudaMemsetAsync(c->fields, 0, 12 * (size_t)ncell * c->tsize, c->stream);
  if (c->tgt) cudaMemsetAsync(c->tgt, 0, 6 * (size_t)ncell * c->tsize, c->stream);
  cudaMemsetAsync(c->J, 0, 3 * (size_t)ncell * sizeof(double), c->stream);
  cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream);
  for (int s = 0; s < kMaxSpecies; ++s) cudaMemsetAsync(c->sp[s].n_dev, 0, sizeof(int), c->stream);
  launch_location_flags(g, c->loc, c->stream);
  if (c->kin) {
    if (c->mixed)
      launch_inner_kappa_table<float>(g, static_cast<float*>(c->kin), c->stream);
    else
      launch_inner_kappa_table<double>(g, static_cast<double*>(c->kin), c->stream);
  }
  grpic_status s = cuda_check(c, cudaGetLastError(), "create");
  if (s == GRPIC_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "create sync");
  if (s != GRPIC_OK) {
    grpic_destroy(c);
    return s;
  }
  *out = c;
  return GRPIC_OK;
}

grpic_status grpic_destroy(grpic_ctx* c) {
  if (!c) return GRPIC_ERR_INVALID;
  cudaStreamSynchronize(c->stream);
  dev_free(c, c->fields);
  dev_free(c, c->tgt);
  dev_free(c, c->kin);
  dev_free(c, c->atab);
  dev_free(c, c->J);
  dev_free(c, c->loc);
  dev_free(c, c->st);
  dev_free(c, c->sort.counts);
  dev_free(c, c->sort.offsets);
  dev_free(c, c->sort.blocks);
  for (int s = 0; s < kMaxSpecies; ++s) {
    dev_free(c, c->inv_e0[s]);
    dev_free(c, c->inv_l0[s]);
    dev_free(c, c->sp[s].buf[0]);
    dev_free(c, c->sp[s].buf[1]);
    dev_free(c, c->sp[s].n_dev);
    dev_free(c, c->sp[s].near_n);
    if (c->sp[s].n_shadow) cudaFreeHost(c->sp[s].n_shadow);
    if (c->sp[s].shadow_ev) cudaEventDestroy(c->sp[s].shadow_ev);
  }
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (auto& p : c->pending) {
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return GRPIC_OK;
}

// Stage a host or device double array on the device; *tmp receives a temporary to free.
static grpic_status stage_in(grpic_ctx* c, const void* src, size_t bytes, int mem, const void** dev, void** tmp) {
  *tmp = nullptr;
  if (mem == GRPIC_MEM_DEVICE) {
    *dev = src;
    return GRPIC_OK;
  }
  void* t = dev_alloc(c, bytes);
  if (!t) return fail(c, GRPIC_ERR_OOM, "staging allocation failed");
  grpic_status s = cuda_check(c, cudaMemcpyAsync(t, src, bytes, cudaMemcpyHostToDevice, c->stream), "H2D copy");
  *tmp = t;
  *dev = t;
  return s;
}

static void release_tmp(grpic_ctx* c, void* tmp) {
  if (!tmp) return;
  cudaStreamSynchronize(c->stream);
  dev_free(c, tmp);
}

grpic_status grpic_set_fields(grpic_ctx* c, const double* d3, const double* b3, int mem) {
  if (!c || !d3 || !b3) return GRPIC_ERR_INVALID;
  const long long n3 = 3 * c->g.ncell;
  const void *dd, *bd;
  void *td, *tb;
  grpic_status s = stage_in(c, d3, sizeof(double) * n3, mem, &dd, &td);
  if (s == GRPIC_OK) s = stage_in(c, b3, sizeof(double) * n3, mem, &bd, &tb);
  if (s != GRPIC_OK) return s;
  // the current buffers (each set of three planes is contiguous)
  if (c->mixed) {
    launch_convert_in<float>(field_plane<float>(c, false, c->dcur, 0), static_cast<const double*>(dd), n3,
                             c->stream);
    launch_convert_in<float>(field_plane<float>(c, true, c->bcur, 0), static_cast<const double*>(bd), n3,
                             c->stream);
  } else {
    cudaMemcpyAsync(field_plane<double>(c, false, c->dcur, 0), dd, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                    c->stream);
    cudaMemcpyAsync(field_plane<double>(c, true, c->bcur, 0), bd, sizeof(double) * n3, cudaMemcpyDeviceToDevice,
                    c->stream);
  }
  snapshot_target(c);
  s = cuda_check(c, cudaGetLastError(), "set_fields");
  release_tmp(c, td);
  release_tmp(c, tb);
  return s;
}

grpic_status grpic_set_uniform_field(grpic_ctx* c, const double E[3], const double B[3]) {
  if (!c || !E || !B) return GRPIC_ERR_INVALID;
  if (c->mixed)
    launch_uniform_field<float>(c->g, fields_view<float>(c), E, B, c->stream);
  else
    launch_uniform_field<double>(c->g, fields_view<double>(c), E, B, c->stream);
  snapshot_target(c);
  grpic_status s = cuda_check(c, cudaGetLastError(), "set_uniform_field");
  if (s == GRPIC_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "set_uniform_field sync");
  return s;
}

grpic_status grpic_set_j(grpic_ctx* c, const double* J3, int mem) {
  if (!c || !J3) return GRPIC_ERR_INVALID;
  const size_t bytes = sizeof(double) * 3 * c->g.ncell;
  grpic_status s = cuda_check(c,
                              cudaMemcpyAsync(c->J, J3, bytes,
                                              mem == GRPIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyHostToDevice,
                                              c->stream),
                              "set_j");
  if (s == GRPIC_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "set_j sync");
  return s;
}

grpic_status grpic_load_particles(grpic_ctx* c, int species, double q_over_m, double q_macro, int64_t n,
                                  const double* x4, const double* u4, const uint32_t* ids, int flags) {
  if (!c || species < 0 || species >= kMaxSpecies || n < 0) return GRPIC_ERR_INVALID;
  if (n > 0 && (!x4 || !u4 || !ids)) return GRPIC_ERR_INVALID;
  if (n >= (1ll << 31) - 1) return fail(c, GRPIC_ERR_CAPACITY, "at most 2^31-2 particles per species");
  const int umode = flags & 3;
  if (umode == 3) return GRPIC_ERR_INVALID;
  const int mem = (flags & GRPIC_LOAD_DEVICE) ? GRPIC_MEM_DEVICE : GRPIC_MEM_HOST;
  grpic_status s = ensure_capacity(c, species, n);
  if (s != GRPIC_OK) return s;
  SpeciesStore& S = c->sp[species];
  const void *xd, *ud, *idd;
  void *tx = nullptr, *tu = nullptr, *ti = nullptr;
  s = stage_in(c, x4, sizeof(double) * 4 * (size_t)n, mem, &xd, &tx);
  if (s == GRPIC_OK) s = stage_in(c, u4, sizeof(double) * 4 * (size_t)n, mem, &ud, &tu);
  if (s == GRPIC_OK) s = stage_in(c, ids, sizeof(uint32_t) * (size_t)n, mem, &idd, &ti);
  if (s != GRPIC_OK) {
    release_tmp(c, tx);
    release_tmp(c, tu);
    release_tmp(c, ti);
    return s;
  }
  S.qm = q_over_m;
  S.qmacro = q_macro;
  S.cur = 0;
  S.n = n;
  S.loaded = true;
  S.shadow_pending = false;
  const double ct_now = c->g.c * c->g.dt * (double)c->pushes;
  const int ni = (int)n;
  cudaMemcpyAsync(S.n_dev, &ni, sizeof(int), cudaMemcpyHostToDevice, c->stream);
  if (c->mixed)
    launch_load_particles<float>(c->g, particles_view<float>(c, species, 0), n, static_cast<const double*>(xd),
                                 static_cast<const double*>(ud), static_cast<const uint32_t*>(idd), umode, ct_now,
                                 c->st, c->stream);
  else
    launch_load_particles<double>(c->g, particles_view<double>(c, species, 0), n, static_cast<const double*>(xd),
                                  static_cast<const double*>(ud), static_cast<const uint32_t*>(idd), umode, ct_now,
                                  c->st, c->stream);
  s = cuda_check(c, cudaGetLastError(), "load_particles");
  // sort once so the store starts cell-ordered
  if (s == GRPIC_OK) {
    if (c->mixed)
      launch_sort<float>(c->g, particles_view<float>(c, species, 0), particles_view<float>(c, species, 1), c->sort,
                         S.n_dev, c->stream);
    else
      launch_sort<double>(c->g, particles_view<double>(c, species, 0), particles_view<double>(c, species, 1),
                          c->sort, S.n_dev, c->stream);
    S.cur = 1;
  }
  if (s == GRPIC_OK) s = read_status(c);
  release_tmp(c, tx);
  release_tmp(c, tu);
  release_tmp(c, ti);
  if (s != GRPIC_OK) {
    S.loaded = false;
    S.n = 0;
  }
  return s;
}

grpic_status grpic_step_async(grpic_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return GRPIC_ERR_INVALID;
  for (int i = 0; i < nsteps; ++i) enqueue_step(c);
  return cuda_check(c, cudaGetLastError(), "step launch");
}

grpic_status grpic_sync(grpic_ctx* c) {
  if (!c) return GRPIC_ERR_INVALID;
  return read_status(c);
}

grpic_status grpic_step(grpic_ctx* c, int nsteps) {
  grpic_status s = grpic_step_async(c, nsteps);
  if (s != GRPIC_OK) return s;
  return read_status(c);
}

grpic_status grpic_stage(grpic_ctx* c, int stage) {
  if (!c || stage < GRPIC_STAGE_B_HALF || stage > GRPIC_STAGE_B_HALF2) return GRPIC_ERR_INVALID;
  enqueue_stage_any(c, stage);
  grpic_status s = cuda_check(c, cudaGetLastError(), "stage launch");
  if (s != GRPIC_OK) return s;
  return read_status(c);
}

grpic_status grpic_get_fields(grpic_ctx* c, double* d3, double* b3, double* J3, int mem) {
  if (!c) return GRPIC_ERR_INVALID;
  const long long n3 = 3 * c->g.ncell;
  const size_t bytes = sizeof(double) * n3;
  const cudaMemcpyKind kind = mem == GRPIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* tmp = nullptr;
  if (c->mixed && (d3 || b3)) {
    tmp = static_cast<double*>(dev_alloc(c, bytes));
    if (!tmp) return fail(c, GRPIC_ERR_OOM, "staging allocation failed");
  }
  double* outs[2] = {d3, b3};
  for (int w = 0; w < 2; ++w) {
    if (!outs[w]) continue;
    const int buf = w ? c->bcur : c->dcur;
    if (c->mixed) {
      launch_convert_out<float>(tmp, field_plane<float>(c, w == 1, buf, 0), n3, c->stream);
      cudaMemcpyAsync(outs[w], tmp, bytes, kind, c->stream);
    } else {
      cudaMemcpyAsync(outs[w], field_plane<double>(c, w == 1, buf, 0), bytes, kind, c->stream);
    }
    cudaStreamSynchronize(c->stream);
  }
  if (J3) cudaMemcpyAsync(J3, c->J, bytes, kind, c->stream);
  grpic_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "get_fields");
  if (tmp) dev_free(c, tmp);
  return s;
}

grpic_status grpic_get_fields_contra(grpic_ctx* c, double* d3, double* h3, int mem) {
  if (!c) return GRPIC_ERR_INVALID;
  grpic_status s = GRPIC_OK;
  if (d3) s = grpic_get_fields(c, d3, nullptr, nullptr, mem);
  if (s != GRPIC_OK || !h3) return s;
  const size_t bytes = sizeof(double) * 3 * c->g.ncell;
  double* out = h3;
  if (mem != GRPIC_MEM_DEVICE) {
    out = static_cast<double*>(dev_alloc(c, bytes));
    if (!out) return fail(c, GRPIC_ERR_OOM, "staging allocation failed");
  }
  if (c->mixed)
    launch_contra_h<float>(c->g, fields_view<float>(c), c->loc, out, c->stream);
  else
    launch_contra_h<double>(c->g, fields_view<double>(c), c->loc, out, c->stream);
  s = cuda_check(c, cudaGetLastError(), "contra_h");
  if (s == GRPIC_OK && out != h3)
    s = cuda_check(c, cudaMemcpyAsync(h3, out, bytes, cudaMemcpyDeviceToHost, c->stream), "contra_h copy");
  if (s == GRPIC_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "contra_h sync");
  if (out != h3) dev_free(c, out);
  return s;
}

// Planes z0 .. z0 + n - 1 of component q of field `which` (the current buffer), as a pointer of T
// (d, b) or double (J); count = n planes of nx * ny.
static bool plane_range_ok(const grpic_ctx* c, int which, int z0, int n) {
  return c && which >= GRPIC_FIELD_D && which <= GRPIC_FIELD_J && z0 >= 0 && n >= 0 && z0 + n <= c->g.nz;
}

grpic_status grpic_get_planes(grpic_ctx* c, int which, int z0, int nplanes, double* buf, int mem) {
  if (!plane_range_ok(c, which, z0, nplanes) || (!buf && nplanes > 0)) return GRPIC_ERR_INVALID;
  const long long plane = (long long)c->g.nx * c->g.ny, count = plane * nplanes;
  if (count == 0) return GRPIC_OK;
  const cudaMemcpyKind kind = mem == GRPIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* tmp = nullptr;
  if (which != GRPIC_FIELD_J && c->mixed) {
    tmp = static_cast<double*>(dev_alloc(c, sizeof(double) * 3 * count));
    if (!tmp) return fail(c, GRPIC_ERR_OOM, "staging allocation failed");
  }
  for (int q = 0; q < 3; ++q) {
    double* dst = buf + q * count;
    if (which == GRPIC_FIELD_J) {
      cudaMemcpyAsync(dst, c->J + (size_t)q * c->g.ncell + z0 * plane, sizeof(double) * count, kind, c->stream);
    } else {
      const bool is_b = which == GRPIC_FIELD_B;
      const int cur = is_b ? c->bcur : c->dcur;
      if (c->mixed) {
        launch_convert_out<float>(tmp + q * count, field_plane<float>(c, is_b, cur, q) + z0 * plane, count,
                                  c->stream);
        cudaMemcpyAsync(dst, tmp + q * count, sizeof(double) * count, kind, c->stream);
      } else {
        cudaMemcpyAsync(dst, field_plane<double>(c, is_b, cur, q) + z0 * plane, sizeof(double) * count, kind,
                        c->stream);
      }
    }
  }
  grpic_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "get_planes");
  if (tmp) dev_free(c, tmp);
  return s;
}

grpic_status grpic_set_planes(grpic_ctx* c, int which, int z0, int nplanes, const double* buf, int mem, int add) {
  if (!plane_range_ok(c, which, z0, nplanes) || (!buf && nplanes > 0) || (add && which != GRPIC_FIELD_J))
    return GRPIC_ERR_INVALID;
  const long long plane = (long long)c->g.nx * c->g.ny, count = plane * nplanes;
  if (count == 0) return GRPIC_OK;
  const void* src;
  void* tmp;
  grpic_status s = stage_in(c, buf, sizeof(double) * 3 * count, mem, &src, &tmp);
  if (s != GRPIC_OK) return s;
  const double* in = static_cast<const double*>(src);
  for (int q = 0; q < 3; ++q) {
    if (which == GRPIC_FIELD_J) {
      double* J = c->J + (size_t)q * c->g.ncell + z0 * plane;
      if (add)
        launch_add_f64(J, in + q * count, count, c->stream);
      else
        cudaMemcpyAsync(J, in + q * count, sizeof(double) * count, cudaMemcpyDeviceToDevice, c->stream);
    } else {
      const bool is_b = which == GRPIC_FIELD_B;
      const int cur = is_b ? c->bcur : c->dcur;
      if (c->mixed)
        launch_convert_in<float>(field_plane<float>(c, is_b, cur, q) + z0 * plane, in + q * count, count, c->stream);
      else
        cudaMemcpyAsync(field_plane<double>(c, is_b, cur, q) + z0 * plane, in + q * count, sizeof(double) * count,
                        cudaMemcpyDeviceToDevice, c->stream);
    }
  }
  s = cuda_check(c, cudaGetLastError(), "set_planes");
  release_tmp(c, tmp);
  if (s == GRPIC_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "set_planes sync");
  return s;
}

grpic_status grpic_num_particles(grpic_ctx* c, int species, int64_t* n) {
  if (!c || !n || species < 0 || species >= kMaxSpecies) return GRPIC_ERR_INVALID;
  SpeciesStore& S = c->sp[species];
  if (!S.loaded) {
    *n = 0;
    return GRPIC_OK;
  }
  int v = 0;
  grpic_status s = cuda_check(c, cudaMemcpyAsync(&v, S.n_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                              "count copy");
  if (s == GRPIC_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "count sync");
  if (s != GRPIC_OK) return s;
  // entries after the last sort may include particles flagged since; sort if needed
  if (c->since_sort != 0) {
    enqueue_stage_any(c, GRPIC_STAGE_SORT);
    c->since_sort = 0;
    s = cuda_check(c, cudaMemcpyAsync(&v, S.n_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "count copy");
    if (s == GRPIC_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "count sync");
    if (s != GRPIC_OK) return s;
  }
  S.n = v;
  S.shadow_pending = false;
  *n = v;
  return GRPIC_OK;
}

grpic_status grpic_get_particles(grpic_ctx* c, int species, int64_t* n_inout, double* x4, double* u4,
                                 uint32_t* ids, int mem) {
  if (!c || !n_inout || species < 0 || species >= kMaxSpecies) return GRPIC_ERR_INVALID;
  int64_t n = 0;
  grpic_status s = grpic_num_particles(c, species, &n);
  if (s != GRPIC_OK) return s;
  if (*n_inout < n) {
    *n_inout = n;
    return fail(c, GRPIC_ERR_CAPACITY, "output arrays too small");
  }
  *n_inout = n;
  if (n == 0) return GRPIC_OK;
  const double ct_now = c->g.c * c->g.dt * (double)c->pushes;
  SpeciesStore& S = c->sp[species];
  double *dx = x4, *du = u4;
  uint32_t* di = ids;
  void *tx = nullptr, *tu = nullptr, *ti = nullptr;
  if (mem != GRPIC_MEM_DEVICE) {
    if (x4) dx = static_cast<double*>(tx = dev_alloc(c, sizeof(double) * 4 * n));
    if (u4) du = static_cast<double*>(tu = dev_alloc(c, sizeof(double) * 4 * n));
    if (ids) di = static_cast<uint32_t*>(ti = dev_alloc(c, sizeof(uint32_t) * n));
    if ((x4 && !tx) || (u4 && !tu) || (ids && !ti)) {
      dev_free(c, tx);
      dev_free(c, tu);
      dev_free(c, ti);
      return fail(c, GRPIC_ERR_OOM, "staging allocation failed");
    }
  }
  if (c->mixed)
    launch_unload_particles<float>(particles_view<float>(c, species, S.cur), n, dx, du, di, ct_now, c->stream);
  else
    launch_unload_particles<double>(particles_view<double>(c, species, S.cur), n, dx, du, di, ct_now, c->stream);
  if (mem != GRPIC_MEM_DEVICE) {
    if (x4) cudaMemcpyAsync(x4, dx, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, c->stream);
    if (u4) cudaMemcpyAsync(u4, du, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, c->stream);
    if (ids) cudaMemcpyAsync(ids, di, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, c->stream);
  }
  s = cuda_check(c, cudaStreamSynchronize(c->stream), "get_particles");
  dev_free(c, tx);
  dev_free(c, tu);
  dev_free(c, ti);
  return s;
}

grpic_status grpic_get_stats(grpic_ctx* c, grpic_stats* out) {
  if (!c || !out) return GRPIC_ERR_INVALID;
  grpic_status s = read_status(c);
  if (s != GRPIC_OK && s != GRPIC_ERR_CFL && s != GRPIC_ERR_NONFINITE) return s;
  *out = c->totals;
  out->steps = c->steps;
  for (int q = 0; q < kMaxSpecies; ++q) {
    int v = 0;
    if (c->sp[q].loaded) {
      cudaMemcpy(&v, c->sp[q].n_dev, sizeof(int), cudaMemcpyDeviceToHost);
    }
    out->n_alive[q] = v;
  }
  return GRPIC_OK;
}

}  // extern "C"

namespace {
template <typename T>
grpic_status invariants(grpic_ctx* c, int set_baseline, grpic_invariants* out) {
  struct Acc {
    unsigned long long n, tracked;
    double norm_sum, e_sum, l_sum;
    unsigned long long norm_max, e_max, l_max;
    unsigned long long max_id;
  };
  if (sizeof(Acc) != invariant_acc_bytes()) return fail(c, GRPIC_ERR_INVALID, "invariant accumulator layout");
  // particles removed since the last sort carry the removed key and are skipped: no sort here, so
  // the call leaves the run's sort schedule as it is
  Acc* acc = static_cast<Acc*>(dev_alloc(c, sizeof(Acc) * (kMaxSpecies + 1)));
  if (!acc) return fail(c, GRPIC_ERR_OOM, "invariant accumulator");
  cudaMemsetAsync(acc, 0, sizeof(Acc) * (kMaxSpecies + 1), c->stream);
  grpic_status st = GRPIC_OK;
  for (int s = 0; s < kMaxSpecies && st == GRPIC_OK; ++s) {
    SpeciesStore& S = c->sp[s];
    if (!S.loaded || S.n == 0) continue;
    const Particles<T> P = particles_view<T>(c, s, S.cur);
    if (set_baseline) {
      launch_max_id<T>(P, &acc[1 + s].max_id, c->stream);
      Acc h{};
      cudaMemcpyAsync(&h, &acc[1 + s], sizeof(Acc), cudaMemcpyDeviceToHost, c->stream);
      st = cuda_check(c, cudaStreamSynchronize(c->stream), "invariants max id");
      if (st != GRPIC_OK) break;
      const long long slots = (long long)(h.max_id / kInvariantStride) + 1;
      if (slots > c->inv_slots[s]) {
        dev_free(c, c->inv_e0[s]);
        dev_free(c, c->inv_l0[s]);
        c->inv_e0[s] = static_cast<double*>(dev_alloc(c, sizeof(double) * slots));
        c->inv_l0[s] = static_cast<double*>(dev_alloc(c, sizeof(double) * slots));
        c->inv_slots[s] = (c->inv_e0[s] && c->inv_l0[s]) ? slots : 0;
        if (!c->inv_slots[s]) st = fail(c, GRPIC_ERR_OOM, "invariant baseline");
      }
      if (st != GRPIC_OK) break;
      // all-ones bytes are a NaN: slots no live particle fills stay untracked
      cudaMemsetAsync(c->inv_e0[s], 0xff, sizeof(double) * c->inv_slots[s], c->stream);
    }
    launch_invariants<T>(c->g, P, set_baseline ? 0 : 1, kInvariantStride, c->inv_e0[s], c->inv_l0[s],
                         c->inv_slots[s], acc, c->stream);
    c->launches += 1;
  }
  Acc h{};
  cudaMemcpyAsync(&h, acc, sizeof(Acc), cudaMemcpyDeviceToHost, c->stream);
  if (st == GRPIC_OK) st = cuda_check(c, cudaStreamSynchronize(c->stream), "invariants");
  else cudaStreamSynchronize(c->stream);
  dev_free(c, acc);
  if (st != GRPIC_OK || !out) return st;
  auto bits = [](unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof(d));
    return d;
  };
  out->n = (int64_t)h.n;
  out->norm_max = bits(h.norm_max);
  out->norm_mean = h.n ? h.norm_sum / (double)h.n : 0.0;
  out->tracked = set_baseline ? 0 : (int64_t)h.tracked;
  out->energy_mean = h.tracked && !set_baseline ? h.e_sum / (double)h.tracked : 0.0;
  out->energy_max = set_baseline ? 0.0 : bits(h.e_max);
  out->angmom_mean = h.tracked && !set_baseline ? h.l_sum / (double)h.tracked : 0.0;
  out->angmom_max = set_baseline ? 0.0 : bits(h.l_max);
  return GRPIC_OK;
}

}  // namespace

extern "C" {

grpic_status grpic_get_invariants(grpic_ctx* c, int set_baseline, grpic_invariants* out) {
  if (!c) return GRPIC_ERR_INVALID;
  return c->mixed ? invariants<float>(c, set_baseline, out) : invariants<double>(c, set_baseline, out);
}

grpic_status grpic_charge_density(grpic_ctx* c, int with_gamma, double* rho, int mem) {
  if (!c || !rho) return GRPIC_ERR_INVALID;
  double* d = rho;
  void* tmp = nullptr;
  if (mem != GRPIC_MEM_DEVICE) {
    d = static_cast<double*>(tmp = dev_alloc(c, sizeof(double) * (size_t)c->g.ncell));
    if (!d) return fail(c, GRPIC_ERR_OOM, "charge density staging");
  }
  if (c->mixed)
    enqueue_rho<float>(c, with_gamma != 0, d);
  else
    enqueue_rho<double>(c, with_gamma != 0, d);
  if (mem != GRPIC_MEM_DEVICE)
    cudaMemcpyAsync(rho, d, sizeof(double) * (size_t)c->g.ncell, cudaMemcpyDeviceToHost, c->stream);
  grpic_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "charge density");
  dev_free(c, tmp);
  return st;
}

grpic_status grpic_gauss_residual(grpic_ctx* c, double* res, int mem, double* max_abs) {
  if (!c || (!res && !max_abs)) return GRPIC_ERR_INVALID;
  const size_t nc = (size_t)c->g.ncell;
  double* rho = static_cast<double*>(dev_alloc(c, sizeof(double) * nc));
  double* r = res;
  void* rtmp = nullptr;
  if (res && mem != GRPIC_MEM_DEVICE) r = static_cast<double*>(rtmp = dev_alloc(c, sizeof(double) * nc));
  unsigned long long* mx = static_cast<unsigned long long*>(dev_alloc(c, sizeof(unsigned long long)));
  if (!rho || !mx || (res && !r)) {
    dev_free(c, rho);
    dev_free(c, rtmp);
    dev_free(c, mx);
    return fail(c, GRPIC_ERR_OOM, "gauss residual staging");
  }
  cudaMemsetAsync(mx, 0, sizeof(unsigned long long), c->stream);
  if (c->mixed) {
    enqueue_rho<float>(c, false, rho);
    launch_gauss<float>(fields_view<float>(c), rho, c->g, 2, r, mx, c->stream);
  } else {
    enqueue_rho<double>(c, false, rho);
    launch_gauss<double>(fields_view<double>(c), rho, c->g, 2, r, mx, c->stream);
  }
  if (res && mem != GRPIC_MEM_DEVICE) cudaMemcpyAsync(res, r, sizeof(double) * nc, cudaMemcpyDeviceToHost, c->stream);
  unsigned long long bits = 0;
  cudaMemcpyAsync(&bits, mx, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
  grpic_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "gauss residual");
  if (st == GRPIC_OK && max_abs) std::memcpy(max_abs, &bits, sizeof(double));
  dev_free(c, rho);
  dev_free(c, rtmp);
  dev_free(c, mx);
  return st;
}

grpic_status grpic_set_tuning(grpic_ctx* c, const grpic_tuning* t) {
  if (!c || !t) return GRPIC_ERR_INVALID;
  if (t->far_min_blocks < 4 || t->far_min_blocks > 6 || t->near_blocks_per_sm < 1 ||
      t->near_blocks_per_sm > 32 || t->sort_interval < 1 || (t->overlap != 0 && t->overlap != 1) ||
      (t->split != 0 && t->split != 1) || (t->j_tile != 0 && t->j_tile != 1) ||
      t->spread < 0 || t->spread > 64 || (t->spread & (t->spread - 1)) != 0 ||
      (t->area_table != 0 && t->area_table != 1))
    return fail(c, GRPIC_ERR_INVALID, "tuning out of range");
  if (t->area_table && t->j_tile) return fail(c, GRPIC_ERR_INVALID, "area_table excludes j_tile");
  if (t->area_table && c->mixed && !c->atab) {
    c->atab = static_cast<float4*>(dev_alloc(c, sizeof(float4) * kAreaTableStride * (size_t)c->g.ncell));
    if (!c->atab) return fail(c, GRPIC_ERR_OOM, "area table allocation");
    launch_area_table(c->g, c->atab, c->stream);
    c->launches += 1;
    const grpic_status s = cuda_check(c, cudaGetLastError(), "area table");
    if (s != GRPIC_OK) return s;
  }
  c->tune = *t;
  c->cfg.sort_interval = t->sort_interval;
  return GRPIC_OK;
}

grpic_status grpic_get_tuning(const grpic_ctx* c, grpic_tuning* t) {
  if (!c || !t) return GRPIC_ERR_INVALID;
  *t = c->tune;
  return GRPIC_OK;
}

grpic_status grpic_set_profiling(grpic_ctx* c, int on) {
  if (!c) return GRPIC_ERR_INVALID;
  c->profiling = on != 0;
  return GRPIC_OK;
}

grpic_status grpic_get_profile(grpic_ctx* c, double times_ms[6], int64_t counts[6], int64_t* kernel_launches,
                               int reset) {
  if (!c) return GRPIC_ERR_INVALID;
  grpic_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "profile sync");
  if (s != GRPIC_OK) return s;
  collect_profile(c);
  for (int q = 0; q < 6; ++q) {
    if (times_ms) times_ms[q] = c->prof_ms[q];
    if (counts) counts[q] = c->prof_cnt[q];
  }
  if (kernel_launches) *kernel_launches = c->launches;
  if (reset) {
    for (int q = 0; q < 6; ++q) {
      c->prof_ms[q] = 0.0;
      c->prof_cnt[q] = 0;
    }
    c->launches = 0;
  }
  return GRPIC_OK;
}

}  // extern "C"

// ---- batched engine ----------------------------------------------------------------------------
struct grpic_batch {
  std::vector<grpic_ctx*> ctxs;
  // the batch's own copy of the device allocator (its tables must be freed with it even after
  // the contexts it was built from are gone)
  grpic_alloc_fn alloc = nullptr;
  grpic_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  cudaStream_t stream = nullptr;  // created by the batch: capturable, ordered with the contexts by events
  bool mixed = false, literal = false;
  int quad = 2;
  std::vector<void*> allocs;
  void* desc = nullptr;
  BlockEntry *btile = nullptr, *etile = nullptr, *all = nullptr, *part = nullptr;
  int nbtile = 0, netile = 0, nall = 0, npart = 0;
  int* dcur = nullptr;  // device d-buffer parity per instance
  int *counts = nullptr, *offsets = nullptr, *tiles = nullptr, *pairs = nullptr, *pair_base = nullptr;
  int* cur = nullptr;  // device ping-pong index per (instance, species)
  long long nbins = 0;
  int npairs = 0;
  int persist_blocks = 0;
  int persist_field_blocks = 0;
  int sms = 1;
  std::vector<long long> pair_n;  // work upper bound of each pair when the batch was built
  // One captured step per step parity k: every step flips each particle store (the sort) and each d
  // buffer (the E step), so replaying graph[k] when each context's (store, d) parity equals its
  // parity at capture XOR k lets the FP32 push run as the single-context kernel per (instance,
  // species), its buffers and constants plain launch parameters.
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::vector<int> cur0, dcur0;  // parities of the contexts when the graphs were captured
  // the per-(instance, species) pushes run on kPushBranches parallel branches of the graph
  static constexpr int kPushBranches = 8;
  cudaStream_t side[kPushBranches] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kPushBranches] = {};
  cudaEvent_t ev = nullptr;
  long long kernels_per_step = 0;
};

namespace {

void* batch_alloc(grpic_batch* b, size_t bytes) {
  void* p = nullptr;
  if (b->alloc) {
    p = b->alloc(bytes, b->alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->allocs.push_back(p);
  return p;
}

void batch_free(grpic_batch* b, void* p) {
  if (!p) return;
  if (b->free_fn)
    b->free_fn(p, b->alloc_user);
  else
    cudaFree(p);
}

template <typename T>
BatchTables<T> batch_tables(grpic_batch* b) {
  BatchTables<T> t;
  t.desc = static_cast<const InstDesc<T>*>(b->desc);
  t.btile = b->btile;
  t.nbtile = b->nbtile;
  t.etile = b->etile;
  t.netile = b->netile;
  t.all = b->all;
  t.nall = b->nall;
  t.part = b->part;
  t.npart = b->npart;
  t.counts = b->counts;
  t.offsets = b->offsets;
  t.tiles = b->tiles;
  t.nbins = b->nbins;
  t.pairs = b->pairs;
  t.npairs = b->npairs;
  t.pair_base = b->pair_base;
  t.persist_blocks = b->persist_blocks;
  t.persist_field_blocks = b->persist_field_blocks;
  return t;
}

void append_blocks(std::vector<BlockEntry>& v, int inst, long long items, int bs) {
  const long long nb = (items + bs - 1) / bs;
  for (long long q = 0; q < nb; ++q) v.push_back(BlockEntry{inst, (int)q});
}

template <typename T>
grpic_status batch_build(grpic_batch* b) {
  const int n = (int)b->ctxs.size();
  std::vector<InstDesc<T>> desc(n);
  std::vector<BlockEntry> btile, etile, all, part;
  std::vector<int> pairs, cur_init, dcur_init(n, 0);
  std::vector<long long> bin_base;
  long long nbins = 0;
  // device ping-pong indices: one int per (instance, species)
  b->cur = static_cast<int*>(batch_alloc(b, sizeof(int) * 4 * n));
  if (!b->cur) return GRPIC_ERR_OOM;
  b->dcur = static_cast<int*>(batch_alloc(b, sizeof(int) * n));
  if (!b->dcur) return GRPIC_ERR_OOM;
  cur_init.assign(4 * n, 0);
  for (int i = 0; i < n; ++i) {
    grpic_ctx* c = b->ctxs[i];
    InstDesc<T>& D = desc[i];
    D.g = c->g;
    D.K32 = field_consts<float>(c->g);
    D.K64 = field_consts<double>(c->g);
    // b[0]: the context's current b (b^{n-1/2} at a step boundary), b[1]: the other buffer
    for (int q = 0; q < 3; ++q) {
      D.FS.d[0][q] = field_plane<T>(c, false, 0, q);
      D.FS.d[1][q] = field_plane<T>(c, false, 1, q);
      D.FS.b[0][q] = field_plane<T>(c, true, c->bcur, q);
      D.FS.b[1][q] = field_plane<T>(c, true, 1 - c->bcur, q);
      D.FS.J[q] = c->J + (size_t)q * c->g.ncell;
    }
    for (int q = 0; q < 6; ++q) D.FS.tgt[q] = target_plane<T>(c, q);
    D.FS.kin = static_cast<const T*>(c->kin);
    D.FS.loc = c->loc;
    D.dcur = b->dcur + i;
    dcur_init[i] = c->dcur;
    D.st = c->st;
    const Grid& g = c->g;
    batch_field_tiles(g, sizeof(T) == sizeof(float), &D.btiles, &D.etiles);
    for (long long q = 0; q < D.btiles.count(); ++q) btile.push_back(BlockEntry{i, (int)q});
    for (long long q = 0; q < D.etiles.count(); ++q) etile.push_back(BlockEntry{i, (int)q});
    append_blocks(all, i, g.ncell, 256);
    for (int s = 0; s < kMaxSpecies; ++s) {
      SpeciesStore& S = c->sp[s];
      SpeciesDesc<T>& SD = D.sp[s];
      SD.active = S.loaded ? 1 : 0;
      SD.qm = S.qm;
      SD.qmacro = S.qmacro;
      SD.C = make_consts<T>(g, Species{S.qm, S.qmacro});
      const double rn = near_radius(g);
      SD.r_near2 = (float)(rn * rn);
      SD.cur = b->cur + 4 * i + s;
      SD.bin_base = 0;
      if (!S.loaded) continue;
      SD.buf[0] = particles_view<T>(c, s, 0);
      SD.buf[1] = particles_view<T>(c, s, 1);
      SD.bin_base = nbins;
      nbins += g.ncell + 1;
      cur_init[4 * i + s] = S.cur;
      pairs.push_back(4 * i + s);
      b->pair_n.push_back(S.n);
      append_blocks(part, 4 * i + s, S.n, 128);
    }
  }
  b->npairs = (int)pairs.size();
  b->nbins = std::max<long long>(nbins, 1);
  b->nbtile = (int)btile.size();
  b->netile = (int)etile.size();
  b->nall = (int)all.size();
  b->npart = (int)part.size();
  b->desc = batch_alloc(b, sizeof(InstDesc<T>) * n);
  b->btile = static_cast<BlockEntry*>(batch_alloc(b, sizeof(BlockEntry) * std::max<size_t>(1, btile.size())));
  b->etile = static_cast<BlockEntry*>(batch_alloc(b, sizeof(BlockEntry) * std::max<size_t>(1, etile.size())));
  b->all = static_cast<BlockEntry*>(batch_alloc(b, sizeof(BlockEntry) * std::max<size_t>(1, all.size())));
  b->part = static_cast<BlockEntry*>(batch_alloc(b, sizeof(BlockEntry) * std::max<size_t>(1, part.size())));
  b->counts = static_cast<int*>(batch_alloc(b, sizeof(int) * b->nbins));
  b->offsets = static_cast<int*>(batch_alloc(b, sizeof(int) * b->nbins));
  b->tiles = static_cast<int*>(batch_alloc(b, sizeof(int) * (scan_tiles(b->nbins) + 1)));
  b->pairs = static_cast<int*>(batch_alloc(b, sizeof(int) * std::max(1, b->npairs)));
  // pair_base: npairs per-step bases, then pair_of_inst for every instance * 4 + species
  b->pair_base = static_cast<int*>(batch_alloc(b, sizeof(int) * (b->npairs + 4 * n)));
  if (!b->desc || !b->btile || !b->etile || !b->all || !b->part || !b->counts || !b->offsets || !b->tiles ||
      !b->pairs || !b->pair_base)
    return GRPIC_ERR_OOM;
  std::vector<int> pair_of_inst(4 * n, 0);
  for (int p = 0; p < b->npairs; ++p) pair_of_inst[pairs[p]] = p;
  cudaStream_t st = b->stream;
  cudaMemcpyAsync(b->desc, desc.data(), sizeof(InstDesc<T>) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b->btile, btile.data(), sizeof(BlockEntry) * btile.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b->etile, etile.data(), sizeof(BlockEntry) * etile.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b->dcur, dcur_init.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b->all, all.data(), sizeof(BlockEntry) * all.size(), cudaMemcpyHostToDevice, st);
  if (!part.empty())
    cudaMemcpyAsync(b->part, part.data(), sizeof(BlockEntry) * part.size(), cudaMemcpyHostToDevice, st);
  if (!pairs.empty()) cudaMemcpyAsync(b->pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b->pair_base + b->npairs, pair_of_inst.data(), sizeof(int) * 4 * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(b->cur, cur_init.data(), sizeof(int) * 4 * n, cudaMemcpyHostToDevice, st);
  return cudaStreamSynchronize(st) == cudaSuccess ? GRPIC_OK : GRPIC_ERR_CUDA;
}

// The FP32-mixed push of a batched step at step parity k (see grpic_batch): per (instance,
// species), the single-context per-warp select kernel over the store the step reads, with the d
// buffer of the step and b^n (the other b buffer, written by the first B half-step).
// The items are spread over the batch's parallel branches, largest first, each to the branch with
// the fewest particles so far, so that small instances run beside large ones.
void batch_enqueue_push_items(grpic_batch* b, int k) {
  struct Item {
    size_t inst;
    int s;
    long long n;
  };
  std::vector<Item> items;
  for (size_t i = 0; i < b->ctxs.size(); ++i)
    for (int s = 0; s < kMaxSpecies; ++s)
      if (b->ctxs[i]->sp[s].loaded && b->ctxs[i]->sp[s].n > 0) items.push_back(Item{i, s, b->ctxs[i]->sp[s].n});
  std::sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.n > y.n; });
  cudaEventRecord(b->ev_fork, b->stream);
  long long load[grpic_batch::kPushBranches] = {};
  for (int br = 0; br < grpic_batch::kPushBranches; ++br) cudaStreamWaitEvent(b->side[br], b->ev_fork, 0);
  for (const Item& it : items) {
    int br = 0;
    for (int q = 1; q < grpic_batch::kPushBranches; ++q)
      if (load[q] < load[br]) br = q;
    load[br] += it.n;
    grpic_ctx* c = b->ctxs[it.inst];
    Fields<float> F;
    for (int q = 0; q < 3; ++q) {
      F.d[q] = field_plane<float>(c, false, b->dcur0[it.inst] ^ k, q);
      F.b[q] = field_plane<float>(c, true, 1 - c->bcur, q);
      F.J[q] = c->J + (size_t)q * c->g.ncell;
    }
    SpeciesStore& S = c->sp[it.s];
    const Particles<float> P = particles_view<float>(c, it.s, b->cur0[4 * it.inst + it.s] ^ k);
    launch_push_select(c->g, F, P, Species{S.qm, S.qmacro}, c->st, c->tune.far_min_blocks, false, c->tune.spread,
                       area_table_of(c), b->side[br]);
  }
  for (int br = 0; br < grpic_batch::kPushBranches; ++br) {
    cudaEventRecord(b->ev_join[br], b->side[br]);
    cudaStreamWaitEvent(b->stream, b->ev_join[br], 0);
  }
}

// One batched timestep (Sec. 2.2 for every instance): B half, J = 0, push + deposit, B half, E,
// removal + sort.  Each field and sort stage is one launch over all instances; the FP32-mixed push
// launches per (instance, species).
template <typename T>
void batch_enqueue_step(grpic_batch* b, int k) {
  const BatchTables<T> t = batch_tables<T>(b);
  launch_batch_b_half<T>(t, 0, b->literal, b->stream);
  launch_batch_zero_j<T>(t, b->stream);
  if constexpr (sizeof(T) == sizeof(float))
    batch_enqueue_push_items(b, k);
  else
    launch_batch_push<T>(t, b->quad, b->stream);
  launch_batch_b_half<T>(t, 1, b->literal, b->stream);
  launch_batch_e_step<T>(t, b->literal, b->stream);
  launch_batch_flip_d<T>(t, (int)b->ctxs.size(), b->stream);
  launch_batch_sort<T>(t, b->stream);
}

}  // namespace

extern "C" {

grpic_status grpic_batch_create(grpic_ctx* const* ctxs, int n, void* stream, grpic_batch** out) {
  (void)stream;
  if (!ctxs || n <= 0 || !out) return GRPIC_ERR_INVALID;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || ctxs[i]->mixed != ctxs[0]->mixed || ctxs[i]->g.quad_order != ctxs[0]->g.quad_order ||
        literal_fields(ctxs[i]) != literal_fields(ctxs[0]))
      return GRPIC_ERR_INVALID;
  grpic_batch* b = new grpic_batch();
  b->ctxs.assign(ctxs, ctxs + n);
  b->alloc = ctxs[0]->cfg.alloc;
  b->free_fn = ctxs[0]->cfg.free_fn;
  b->alloc_user = ctxs[0]->cfg.alloc_user;
  b->mixed = ctxs[0]->mixed;
  b->quad = ctxs[0]->g.quad_order;
  b->literal = literal_fields(ctxs[0]);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->sms = std::max(1, sms);
  b->persist_blocks = b->sms * 8;
  b->persist_field_blocks = b->sms * 2;
  bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int br = 0; br < grpic_batch::kPushBranches && ok; ++br)
    ok = cudaStreamCreateWithFlags(&b->side[br], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_join[br], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    grpic_batch_destroy(b);
    return GRPIC_ERR_CUDA;
  }
  for (grpic_ctx* c : b->ctxs) cudaStreamSynchronize(c->stream);
  const grpic_status s = b->mixed ? batch_build<float>(b) : batch_build<double>(b);
  if (s != GRPIC_OK) {
    grpic_batch_destroy(b);
    return s;
  }
  // kernels per step: B halves 2, zero J 1, push (FP32-mixed: one per pair; FP64: 1), E 1, d parity 1,
  // sort 5 (+2 with particles; and 1 memset)
  const int push_launches = b->npart > 0 ? (b->mixed ? b->npairs : 1) : 0;
  b->kernels_per_step = 2 + 1 + push_launches + 1 + 1 + (b->npairs ? 5 + 2 * (b->npart > 0 ? 1 : 0) : 0);
  *out = b;
  return GRPIC_OK;
}

grpic_status grpic_batch_step(grpic_batch* b, int nsteps) {
  if (!b || nsteps < 0) return GRPIC_ERR_INVALID;
  // the batch was built for the particle counts of its creation
  size_t p = 0;
  for (grpic_ctx* c : b->ctxs)
    for (int s = 0; s < kMaxSpecies; ++s)
      if (c->sp[s].loaded && (p >= b->pair_n.size() || c->sp[s].n > b->pair_n[p++])) return GRPIC_ERR_INVALID;
  // order after each context's pending work; refresh the device ping-pong indices
  std::vector<int> cur(4 * b->ctxs.size(), 0);
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    grpic_ctx* c = b->ctxs[i];
    for (int s = 0; s < kMaxSpecies; ++s) cur[4 * i + s] = c->sp[s].cur;
    cudaEventRecord(b->ev, c->stream);
    cudaStreamWaitEvent(b->stream, b->ev, 0);
  }
  cudaMemcpyAsync(b->cur, cur.data(), sizeof(int) * cur.size(), cudaMemcpyHostToDevice, b->stream);
  std::vector<int> dpar(b->ctxs.size(), 0);
  for (size_t i = 0; i < b->ctxs.size(); ++i) dpar[i] = b->ctxs[i]->dcur;
  cudaMemcpyAsync(b->dcur, dpar.data(), sizeof(int) * dpar.size(), cudaMemcpyHostToDevice, b->stream);
  // the step parity of the contexts relative to the captured graphs (recaptured when a context
  // was stepped on its own so that its parities no longer follow the batch's)
  int k = -1;
  if (b->graph[0] && b->graph[1]) {
    for (int kk = 0; kk < 2 && k < 0; ++kk) {
      bool ok = true;
      for (size_t i = 0; i < b->ctxs.size() && ok; ++i) {
        ok = b->ctxs[i]->dcur == (b->dcur0[i] ^ kk);
        for (int s = 0; s < kMaxSpecies && ok; ++s)
          if (b->ctxs[i]->sp[s].loaded) ok = b->ctxs[i]->sp[s].cur == (b->cur0[4 * i + s] ^ kk);
      }
      if (ok) k = kk;
    }
  }
  if (k < 0) {
    for (int kk = 0; kk < 2; ++kk)
      if (b->graph[kk]) {
        cudaGraphExecDestroy(b->graph[kk]);
        b->graph[kk] = nullptr;
      }
    b->cur0 = cur;
    b->dcur0 = dpar;
    for (int kk = 0; kk < 2; ++kk) {
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GRPIC_ERR_CUDA;
      if (b->mixed)
        batch_enqueue_step<float>(b, kk);
      else
        batch_enqueue_step<double>(b, kk);
      if (cudaStreamEndCapture(b->stream, &graph) != cudaSuccess || !graph) return GRPIC_ERR_CUDA;
      const cudaError_t e = cudaGraphInstantiate(&b->graph[kk], graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return GRPIC_ERR_CUDA;
    }
    k = 0;
  }
  for (int j = 0; j < nsteps; ++j)
    if (cudaGraphLaunch(b->graph[(k + j) & 1], b->stream) != cudaSuccess) return GRPIC_ERR_CUDA;
  cudaMemcpyAsync(cur.data(), b->cur, sizeof(int) * cur.size(), cudaMemcpyDeviceToHost, b->stream);
  std::vector<int> dcur(b->ctxs.size(), 0);
  cudaMemcpyAsync(dcur.data(), b->dcur, sizeof(int) * dcur.size(), cudaMemcpyDeviceToHost, b->stream);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return GRPIC_ERR_CUDA;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    grpic_ctx* c = b->ctxs[i];
    c->steps += nsteps;
    c->pushes += nsteps;
    c->since_sort = 0;
    c->dcur = dcur[i];
    c->launches += (long long)nsteps * b->kernels_per_step / (long long)b->ctxs.size();
    for (int s = 0; s < kMaxSpecies; ++s) {
      c->sp[s].cur = cur[4 * i + s];
      c->sp[s].shadow_pending = false;
    }
  }
  // every context's status is read (and kept in its step_status), so one failed instance does
  // not hide the state of the others; the first error is returned
  grpic_status first = GRPIC_OK;
  for (grpic_ctx* c : b->ctxs) {
    c->step_status = read_status(c);
    if (first == GRPIC_OK) first = c->step_status;
  }
  return first;
}

grpic_status grpic_batch_ctx_status(const grpic_ctx* c) { return c ? c->step_status : GRPIC_ERR_INVALID; }

grpic_status grpic_batch_set_blocks_per_sm(grpic_batch* b, int blocks_per_sm) {
  if (!b || blocks_per_sm < 1 || blocks_per_sm > 32) return GRPIC_ERR_INVALID;
  if (b->persist_blocks == b->sms * blocks_per_sm) return GRPIC_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  b->persist_blocks = b->sms * blocks_per_sm;
  for (int kk = 0; kk < 2; ++kk)
    if (b->graph[kk]) {
      cudaGraphExecDestroy(b->graph[kk]);
      b->graph[kk] = nullptr;  // re-captured with the new grid by the next grpic_batch_step
    }
  return GRPIC_OK;
}

grpic_status grpic_batch_info(grpic_batch* b, int64_t* kernels_per_step, int64_t* work_blocks) {
  if (!b) return GRPIC_ERR_INVALID;
  if (kernels_per_step) *kernels_per_step = b->kernels_per_step;
  if (work_blocks) *work_blocks = (int64_t)b->nbtile + b->netile + b->nall + b->npart;
  return GRPIC_OK;
}

grpic_status grpic_batch_destroy(grpic_batch* b) {
  if (!b) return GRPIC_ERR_INVALID;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int kk = 0; kk < 2; ++kk)
    if (b->graph[kk]) cudaGraphExecDestroy(b->graph[kk]);
  for (void* p : b->allocs) batch_free(b, p);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (int br = 0; br < grpic_batch::kPushBranches; ++br) {
    if (b->ev_join[br]) cudaEventDestroy(b->ev_join[br]);
    if (b->side[br]) cudaStreamDestroy(b->side[br]);
  }
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return GRPIC_OK;
}

}  // extern "C"
