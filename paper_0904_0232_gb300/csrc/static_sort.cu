// Cell sort of a particle set without any device allocation.
//
// This is the library's counting sort by cell (histogram -> prefix sum -> scatter) as a
// standalone call whose scratch (per-cell counts, offsets and the prefix-sum tile totals)
// lives in one file-scope __device__ array instead of memory the library allocates.  It is
// for callers that cannot allocate device memory at the point of the call: code that runs
// under a fixed, pre-reserved device-memory budget, code called from inside a memory-pool or
// allocator callback (where allocating again would re-enter the allocator), or a hot loop
// that must never block in cudaMalloc / cudaFree.  The caller provides inputs and outputs.
//
// Every GPU that loads the library holds the array (kMaxCells + 1 counts, as many offsets,
// and the tile totals: about 2.1 MB) until the process exits.  All calls share it and it
// keeps the last call's contents, so each call clears the counts it uses; two calls whose
// work overlaps on the GPU (different streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/grpic.h"

namespace {

constexpr long long kMaxCells = 262144;  // grids of at most 64^3 cells
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr long long kMaxBins = kMaxCells + 1;  // + one bin for particles outside the grid
constexpr int kMaxTiles = (int)((kMaxBins + kTile - 1) / kTile);
constexpr long long kScratchInts = 2 * kMaxBins + kMaxTiles;

static __device__ __align__(256) int g_scratch[kScratchInts];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
int* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (resolved once per device).
grpic_status scratch_address(int** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GRPIC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return GRPIC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<int*>(p);
  }
  *out = g_scratch_ptr[dev];
  return GRPIC_OK;
}

struct Dims {
  int nx, ny, nz;
};

// Cell of a particle, or the outside bin when its position is not inside [0, n-1) per axis.
__device__ __forceinline__ long long cell_of(const Dims& g, const double* x4, long long n, long long i) {
  const double x = x4[i], y = x4[n + i], z = x4[2 * n + i];
  if (!(x >= 0.0 && x < g.nx - 1) || !(y >= 0.0 && y < g.ny - 1) || !(z >= 0.0 && z < g.nz - 1))
    return (long long)g.nx * g.ny * g.nz;
  return ((long long)floor(z) * g.ny + (long long)floor(y)) * g.nx + (long long)floor(x);
}

__global__ void k_count(Dims g, const double* __restrict__ x4, long long n, int* __restrict__ counts) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(counts + cell_of(g, x4, n, i), 1);
}

__device__ __forceinline__ int block_scan(int v, int* ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) ws[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < kThreads / 32) ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < kThreads / 32) ws[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += ws[wid - 1];
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kThreads) k_tile_totals(const int* __restrict__ in, long long n,
                                                            int* __restrict__ tiles) {
  __shared__ int ws[kThreads / 32];
  const long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
  int s = 0;
#pragma unroll
  for (int q = 0; q < kItems; ++q)
    if (base + q < n) s += in[base + q];
  const int inc = block_scan(s, ws);
  if (threadIdx.x == kThreads - 1) tiles[blockIdx.x] = inc;
}

__global__ void __launch_bounds__(kThreads) k_tile_offsets(int* __restrict__ tiles, int ntiles) {
  __shared__ int ws[kThreads / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += kThreads) {
    const int idx = base + threadIdx.x;
    const int v = idx < ntiles ? tiles[idx] : 0;
    const int inc = block_scan(v, ws);
    const int c0 = carry;
    if (idx < ntiles) tiles[idx] = c0 + inc - v;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = c0 + inc;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) k_offsets(const int* __restrict__ in, long long n,
                                                        const int* __restrict__ tiles, int* __restrict__ out) {
  __shared__ int ws[kThreads / 32];
  const long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
  int v[kItems];
  int s = 0;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0;
    s += v[q];
  }
  const int inc = block_scan(s, ws);
  int run = tiles[blockIdx.x] + inc - s;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
}

__global__ void k_place(Dims g, const double* __restrict__ x4, const double* __restrict__ u4,
                        const uint32_t* __restrict__ ids, long long n, int* __restrict__ cursor,
                        double* __restrict__ xo, double* __restrict__ uo, uint32_t* __restrict__ io) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long c = cell_of(g, x4, n, i);
  if (c == (long long)g.nx * g.ny * g.nz) return;
  const long long p = atomicAdd(cursor + c, 1);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    xo[q * n + p] = x4[q * n + i];
    uo[q * n + p] = u4[q * n + i];
  }
  io[p] = ids[i];
}

__global__ void k_kept(const int* __restrict__ offsets, long long outside_bin, int64_t* __restrict__ n_out) {
  *n_out = offsets[outside_bin];
}

}  // namespace

extern "C" grpic_status grpic_sort_particles_static(int nx, int ny, int nz, int64_t n, const double* x4,
                                                    const double* u4, const uint32_t* ids, double* x4_out,
                                                    double* u4_out, uint32_t* ids_out, int64_t* n_out,
                                                    void* stream) {
  if (nx < 2 || ny < 2 || nz < 2 || n < 0 || !n_out) return GRPIC_ERR_INVALID;
  if (n > 0 && (!x4 || !u4 || !ids || !x4_out || !u4_out || !ids_out)) return GRPIC_ERR_INVALID;
  const long long ncell = (long long)nx * ny * nz;
  if (ncell > kMaxCells || n >= (1ll << 31)) return GRPIC_ERR_CAPACITY;
  int* scratch = nullptr;
  grpic_status s = scratch_address(&scratch);
  if (s != GRPIC_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long nbins = ncell + 1;
  const int ntiles = (int)((nbins + kTile - 1) / kTile);
  int* counts = scratch;
  int* offsets = scratch + kMaxBins;
  int* tiles = scratch + 2 * kMaxBins;
  const Dims g{nx, ny, nz};
  // the array keeps the previous call's contents: the counts must start at zero
  if (cudaMemsetAsync(counts, 0, sizeof(int) * nbins, st) != cudaSuccess) return GRPIC_ERR_CUDA;
  const unsigned nb = (unsigned)((n + 255) / 256);
  if (n > 0) k_count<<<nb, 256, 0, st>>>(g, x4, n, counts);
  k_tile_totals<<<ntiles, kThreads, 0, st>>>(counts, nbins, tiles);
  k_tile_offsets<<<1, kThreads, 0, st>>>(tiles, ntiles);
  k_offsets<<<ntiles, kThreads, 0, st>>>(counts, nbins, tiles, offsets);
  if (n > 0) k_place<<<nb, 256, 0, st>>>(g, x4, u4, ids, n, offsets, x4_out, u4_out, ids_out);
  k_kept<<<1, 1, 0, st>>>(offsets, ncell, n_out);
  return cudaGetLastError() == cudaSuccess ? GRPIC_OK : GRPIC_ERR_CUDA;
}
