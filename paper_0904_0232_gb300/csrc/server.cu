// Request serving over whole GRPIC runs (not in the paper): admission by device-memory budget
// and slots, device-side plasma generation per admitted run, one batched timestep per tick over
// every running run (continuous batching), retirement of finished runs.
//
// The plasma generator draws from a counter-based hash (the SplitMix64 finaliser of Steele, Lea
// and Flood) keyed by (seed, stream, counter): positions uniform in each cell of [1, n-3]^3,
// covariant spatial momenta with Maxwell-Juettner magnitudes (inverse-CDF table) and isotropic
// directions.  u^4 is completed by the regular load path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "../../include/grpic.h"

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform in [0, 1) from (seed, stream, counter)
__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long stream,
                                            unsigned long long counter) {
  const unsigned long long h = mix64(mix64(seed) ^ mix64(stream + 0x632BE59BD9B4E019ull) ^ counter);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

constexpr int kTable = 4096;

struct GenParams {
  int nx, ny, nz;
  int ppc, nspecies;
  double xc, yc, zc, r_min2, c;
  unsigned long long seed;
};

// One thread per (cell, slot); kept particles are compacted with an atomic counter and keep
// their slot index as id, so the particle set does not depend on the order.  With x4 == NULL
// the kernel only counts; otherwise the planes have stride `stride` (the kept count).
__global__ void k_generate(GenParams p, const double* __restrict__ inv_cdf, double* __restrict__ x4,
                           double* __restrict__ u4, unsigned* __restrict__ ids, long long stride,
                           unsigned long long* __restrict__ kept) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long wx = p.nx - 3, wy = p.ny - 3;
  const long long ncell = wx * wy * (long long)(p.nz - 3);
  if (t >= ncell * p.ppc) return;
  const long long cell = t / p.ppc;
  const int i = 1 + (int)(cell % wx);
  const int j = 1 + (int)((cell / wx) % wy);
  const int k = 1 + (int)(cell / (wx * wy));
  const double x = i + uniform01(p.seed, 0, 3 * t);
  const double y = j + uniform01(p.seed, 0, 3 * t + 1);
  const double z = k + uniform01(p.seed, 0, 3 * t + 2);
  const double dx = x - p.xc, dy = y - p.yc, dz = z - p.zc;
  if (dx * dx + dy * dy + dz * dz < p.r_min2) return;
  const long long w = (long long)atomicAdd(kept, 1ull);
  if (!x4 || w >= stride) return;
  const long long nmax = stride;
  x4[w] = x;
  x4[nmax + w] = y;
  x4[2 * nmax + w] = z;
  x4[3 * nmax + w] = 0.0;
  ids[w] = (unsigned)t;
  for (int s = 0; s < p.nspecies; ++s) {
    const unsigned long long st = 1 + (unsigned long long)s;
    const double q = uniform01(p.seed, st, 3 * t) * (kTable - 1);
    const int qi = min((int)q, kTable - 2);
    const double mag = inv_cdf[qi] + (q - qi) * (inv_cdf[qi + 1] - inv_cdf[qi]);
    const double ct = 2.0 * uniform01(p.seed, st, 3 * t + 1) - 1.0;
    const double ph = 6.283185307179586 * uniform01(p.seed, st, 3 * t + 2);
    const double sn = sqrt(fmax(0.0, 1.0 - ct * ct));
    double* u = u4 + (size_t)s * 4 * nmax;
    u[w] = p.c * mag * sn * cos(ph);
    u[nmax + w] = p.c * mag * sn * sin(ph);
    u[2 * nmax + w] = p.c * mag * ct;
    u[3 * nmax + w] = 0.0;
  }
}

// Inverse CDF of |u| (units of c) for f(u) ~ u^2 exp(-(sqrt(1+u^2) - 1)/theta), sampled on a
// uniform probability grid of kTable points.
std::vector<double> mj_inverse_cdf(double theta) {
  const int n = 20001;
  const double umax = std::sqrt((1.0 + 40.0 * theta) * (1.0 + 40.0 * theta) - 1.0);
  std::vector<double> u(n), cdf(n, 0.0);
  for (int q = 0; q < n; ++q) u[q] = umax * q / (n - 1);
  auto pdf = [&](double v) { return v * v * std::exp(-(std::sqrt(1.0 + v * v) - 1.0) / theta); };
  for (int q = 1; q < n; ++q) cdf[q] = cdf[q - 1] + 0.5 * (pdf(u[q]) + pdf(u[q - 1])) * (u[q] - u[q - 1]);
  for (int q = 0; q < n; ++q) cdf[q] /= cdf[n - 1];
  std::vector<double> inv(kTable);
  int q = 0;
  for (int r = 0; r < kTable; ++r) {
    const double P = (double)r / (kTable - 1);
    while (q < n - 2 && cdf[q + 1] < P) ++q;
    const double span = cdf[q + 1] - cdf[q];
    inv[r] = span > 0 ? u[q] + (P - cdf[q]) / span * (u[q + 1] - u[q]) : u[q];
  }
  return inv;
}

// Admission limits of the field update's outer boundary (see grpic_submit in include/grpic.h).
constexpr double kMaxFaceF = 0.2;
constexpr double kMaxUnstableTime = 40.0;

long long interior_slots(const grpic_request& r) {
  return (long long)(r.cfg.nx - 3) * (r.cfg.ny - 3) * (r.cfg.nz - 3) * r.ppc;
}

struct Run {
  uint64_t ticket = 0;
  grpic_request req{};
  grpic_ctx* ctx = nullptr;
  int remaining = 0;
  int state = GRPIC_RUN_QUEUED;
  grpic_status err = GRPIC_OK;
  size_t bytes = 0;
};

}  // namespace

struct grpic_server {
  size_t budget = 0, used = 0;
  int max_slots = 1;
  grpic_alloc_fn alloc = nullptr;
  grpic_free_fn free_fn = nullptr;
  void* user = nullptr;
  cudaStream_t stream = nullptr;
  std::deque<Run*> queue;
  std::vector<Run*> running;
  std::map<uint64_t, Run*> runs;
  grpic_batch* batch = nullptr;
  bool dirty = false;
  uint64_t next_ticket = 1;
  bool have_kind = false;
  int precision = 0, quad = 0;
  unsigned flags = 0;
};

namespace {

void* s_alloc(grpic_server* s, size_t bytes) {
  if (s->alloc) return s->alloc(bytes, s->user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void s_free(grpic_server* s, void* p) {
  if (!p) return;
  if (s->free_fn)
    s->free_fn(p, s->user);
  else
    cudaFree(p);
}

// Create the run's context, set its field and generate + load its plasma.
grpic_status start_run(grpic_server* s, Run* r) {
  grpic_config cfg = r->req.cfg;
  cfg.alloc = s->alloc;
  cfg.free_fn = s->free_fn;
  cfg.alloc_user = s->user;
  cfg.sort_interval = 1;
  grpic_status st = grpic_create(&cfg, s->stream, &r->ctx);
  if (st != GRPIC_OK) return st;
  st = grpic_set_uniform_field(r->ctx, r->req.E_contra, r->req.B_contra);
  if (st != GRPIC_OK) return st;
  const long long nmax = interior_slots(r->req);
  const int nsp = r->req.nspecies;
  double* x4 = static_cast<double*>(s_alloc(s, sizeof(double) * 4 * (size_t)std::max(1ll, nmax)));
  double* u4 = static_cast<double*>(s_alloc(s, sizeof(double) * 4 * (size_t)std::max(1ll, nmax) * nsp));
  unsigned* ids = static_cast<unsigned*>(s_alloc(s, sizeof(unsigned) * (size_t)std::max(1ll, nmax)));
  double* table = static_cast<double*>(s_alloc(s, sizeof(double) * kTable));
  unsigned long long* kept = static_cast<unsigned long long*>(s_alloc(s, sizeof(unsigned long long)));
  if (!x4 || !u4 || !ids || !table || !kept) st = GRPIC_ERR_OOM;
  if (st == GRPIC_OK) {
    const double theta = (r->req.u_th / cfg.c) * (r->req.u_th / cfg.c);
    const std::vector<double> inv = mj_inverse_cdf(std::max(theta, 1e-8));
    cudaMemcpyAsync(table, inv.data(), sizeof(double) * kTable, cudaMemcpyHostToDevice, s->stream);
    cudaMemsetAsync(kept, 0, sizeof(unsigned long long), s->stream);
    GenParams gp{cfg.nx, cfg.ny, cfg.nz, r->req.ppc, nsp, 0.5 * (cfg.nx - 1), 0.5 * (cfg.ny - 1),
                 0.5 * (cfg.nz - 1), r->req.r_min * r->req.r_min, cfg.c, (unsigned long long)r->req.seed};
    const unsigned nb = (unsigned)((nmax + 255) / 256);
    unsigned long long n = 0;
    if (nmax > 0) {
      // pass 1: count the kept particles; pass 2: write them with plane stride n
      k_generate<<<nb, 256, 0, s->stream>>>(gp, table, nullptr, nullptr, nullptr, 0, kept);
      cudaMemcpyAsync(&n, kept, sizeof(n), cudaMemcpyDeviceToHost, s->stream);
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) st = GRPIC_ERR_CUDA;
      cudaMemsetAsync(kept, 0, sizeof(unsigned long long), s->stream);
      if (st == GRPIC_OK && n > 0)
        k_generate<<<nb, 256, 0, s->stream>>>(gp, table, x4, u4, ids, (long long)n, kept);
      if (cudaStreamSynchronize(s->stream) != cudaSuccess) st = GRPIC_ERR_CUDA;
    }
    for (int sp = 0; sp < nsp && st == GRPIC_OK; ++sp)
      st = grpic_load_particles(r->ctx, sp, r->req.q_over_m[sp], r->req.q_macro[sp], (int64_t)n,
                                u4 == nullptr ? nullptr : x4, u4 + (size_t)sp * 4 * n,
                                reinterpret_cast<const uint32_t*>(ids), GRPIC_U_COV_SPATIAL | GRPIC_LOAD_DEVICE);
  }
  cudaStreamSynchronize(s->stream);
  // invariant baseline of the run's initial plasma (reported at completion)
  if (st == GRPIC_OK) st = grpic_get_invariants(r->ctx, 1, nullptr);
  s_free(s, x4);
  s_free(s, u4);
  s_free(s, ids);
  s_free(s, table);
  s_free(s, kept);
  return st;
}

}  // namespace

extern "C" {

grpic_status grpic_request_bytes(const grpic_request* r, size_t* bytes) {
  if (!r || !bytes) return GRPIC_ERR_INVALID;
  const double cells = (double)r->cfg.nx * r->cfg.ny * r->cfg.nz;
  const double tsz = r->cfg.precision == GRPIC_FP32_MIXED ? 4.0 : 8.0;
  const double n = (double)interior_slots(*r);
  // 12 field planes (two d and two b buffers; 6 more for the absorbing layers' target), FP64 J,
  // location flags, sort counts and offsets
  const bool layers = r->cfg.absorb_inner > 0.0 || r->cfg.absorb_outer > 0.0;
  const double fields = cells * ((layers ? 18.0 : 12.0) * tsz + 3.0 * 8.0 + 2.0 + 8.0);
  const double particles = n * r->nspecies * 2.0 * (8.0 * tsz + 8.0);
  const double staging = n * (4.0 * 8.0 * (1 + r->nspecies) + 4.0);
  *bytes = (size_t)(fields + particles + staging) + (size_t)(1 << 20);
  return GRPIC_OK;
}

grpic_status grpic_server_create(size_t hbm_budget, int max_slots, grpic_alloc_fn alloc, grpic_free_fn free_fn,
                                 void* alloc_user, grpic_server** out) {
  if (!out || max_slots <= 0 || (alloc == nullptr) != (free_fn == nullptr)) return GRPIC_ERR_INVALID;
  grpic_server* s = new grpic_server();
  s->budget = hbm_budget;
  s->max_slots = max_slots;
  s->alloc = alloc;
  s->free_fn = free_fn;
  s->user = alloc_user;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return GRPIC_ERR_CUDA;
  }
  *out = s;
  return GRPIC_OK;
}

grpic_status grpic_submit(grpic_server* s, const grpic_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket || req->nspecies < 1 || req->nspecies > 4 || req->ppc < 0 || req->nsteps < 0 ||
      req->cfg.nx < 8 || req->cfg.ny < 8 || req->cfg.nz < 8 || req->cfg.z_origin != 0 ||
      (req->cfg.nz_total != 0 && req->cfg.nz_total != req->cfg.nz))
    return GRPIC_ERR_INVALID;  // (a served run is a whole grid)
  const int quad = req->cfg.quad_order == 0 ? 2 : req->cfg.quad_order;
  if (s->have_kind && (req->cfg.precision != s->precision || quad != s->quad || req->cfg.flags != s->flags))
    return GRPIC_ERR_INVALID;
  // the box's faces where f = 2m / R_face > 0.2: with frozen faces the field update grows an edge
  // mode there (measured onset ~40 light-crossing units), so long runs on such grids are refused
  // unless the request has an outer absorbing layer
  const int nmin = std::min(req->cfg.nx, std::min(req->cfg.ny, req->cfg.nz));
  const double f_face = 2.0 * req->cfg.m / (0.5 * (nmin - 1));
  if (f_face > kMaxFaceF && (double)req->nsteps * req->cfg.c * req->cfg.dt > kMaxUnstableTime &&
      !(req->cfg.absorb_outer > 0.0))
    return GRPIC_ERR_UNSTABLE;
  size_t bytes = 0;
  grpic_request_bytes(req, &bytes);
  if (bytes > s->budget) return GRPIC_ERR_CAPACITY;
  if (!s->have_kind) {
    s->have_kind = true;
    s->precision = req->cfg.precision;
    s->quad = quad;
    s->flags = req->cfg.flags;
  }
  Run* r = new Run();
  r->ticket = s->next_ticket++;
  r->req = *req;
  r->remaining = req->nsteps;
  r->bytes = bytes;
  s->queue.push_back(r);
  s->runs[r->ticket] = r;
  *ticket = r->ticket;
  return GRPIC_OK;
}

grpic_status grpic_server_tick(grpic_server* s, int* running, int* queued) {
  if (!s) return GRPIC_ERR_INVALID;
  grpic_status result = GRPIC_OK;
  // admission, in arrival order
  while (!s->queue.empty() && (int)s->running.size() < s->max_slots && s->used + s->queue.front()->bytes <= s->budget) {
    Run* r = s->queue.front();
    s->queue.pop_front();
    s->used += r->bytes;
    r->err = start_run(s, r);
    if (r->err != GRPIC_OK || r->remaining == 0) {
      r->state = GRPIC_RUN_DONE;
      continue;
    }
    r->state = GRPIC_RUN_RUNNING;
    s->running.push_back(r);
    s->dirty = true;
  }
  if (!s->running.empty()) {
    if (s->dirty) {
      if (s->batch) grpic_batch_destroy(s->batch);
      s->batch = nullptr;
      std::vector<grpic_ctx*> ctxs;
      for (Run* r : s->running) ctxs.push_back(r->ctx);
      result = grpic_batch_create(ctxs.data(), (int)ctxs.size(), nullptr, &s->batch);
      s->dirty = false;
    }
    bool batch_ok = result == GRPIC_OK;
    if (batch_ok) {
      const grpic_status st = grpic_batch_step(s->batch, 1);
      // instance errors are per run; anything else (a CUDA error) fails every running run
      batch_ok = st == GRPIC_OK || st == GRPIC_ERR_CFL || st == GRPIC_ERR_NONFINITE || st == GRPIC_ERR_INVALID;
      if (!batch_ok) result = st;
    }
    std::vector<Run*> still;
    for (Run* r : s->running) {
      r->remaining -= 1;
      const grpic_status own = batch_ok ? grpic_batch_ctx_status(r->ctx) : result;
      if (own != GRPIC_OK) r->err = own;
      if (r->remaining <= 0 || own != GRPIC_OK) {
        r->state = GRPIC_RUN_DONE;
        s->dirty = true;
      } else {
        still.push_back(r);
      }
    }
    s->running.swap(still);
    // a batch built over runs that have now finished refers to contexts the caller may release
    // before the next tick: drop it now (the next tick builds one over the running runs)
    if ((s->dirty || s->running.empty()) && s->batch) {
      grpic_batch_destroy(s->batch);
      s->batch = nullptr;
    }
  }
  if (running) *running = (int)s->running.size();
  if (queued) *queued = (int)s->queue.size();
  return result;
}

grpic_status grpic_poll(grpic_server* s, uint64_t ticket, int* state, grpic_ctx** ctx) {
  if (!s || !state) return GRPIC_ERR_INVALID;
  auto it = s->runs.find(ticket);
  if (it == s->runs.end()) return GRPIC_ERR_INVALID;
  Run* r = it->second;
  *state = r->state;
  if (ctx) *ctx = r->state == GRPIC_RUN_DONE ? r->ctx : nullptr;
  return r->state == GRPIC_RUN_DONE ? r->err : GRPIC_ERR_AGAIN;
}

grpic_status grpic_server_release(grpic_server* s, uint64_t ticket) {
  if (!s) return GRPIC_ERR_INVALID;
  auto it = s->runs.find(ticket);
  if (it == s->runs.end() || it->second->state != GRPIC_RUN_DONE) return GRPIC_ERR_INVALID;
  Run* r = it->second;
  if (r->ctx) grpic_destroy(r->ctx);
  s->used -= r->bytes;
  s->runs.erase(it);
  delete r;
  return GRPIC_OK;
}

grpic_status grpic_server_destroy(grpic_server* s) {
  if (!s) return GRPIC_ERR_INVALID;
  if (s->batch) grpic_batch_destroy(s->batch);
  for (auto& kv : s->runs) {
    if (kv.second->ctx) grpic_destroy(kv.second->ctx);
    delete kv.second;
  }
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return GRPIC_OK;
}

}  // extern "C"
