// Particle removal and counting sort by cell (not in the paper: the paper names no boundary
// treatment; removed particles carry key kDead and are dropped here).
//
//   1. histogram of the keys into ncell + 1 bins (the last bin collects removed particles);
//   2. exclusive prefix sum of the bins (block-level warp-shuffle scans, three passes);
//   3. scatter of x, u, id, key into the alternate buffers at bin offset + running count.
// The live count (start of the removed bin) is left in device memory, so no host round
// trip is needed between steps.  Within a cell the order is not stable.
#include "common.cuh"

namespace grpic {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_hist(const uint32_t* __restrict__ key, long long n, const int* __restrict__ n_dev,
                       int* __restrict__ counts, long long dead_bin) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n || i >= (long long)(*n_dev)) return;
  const uint32_t k = key[i];
  atomicAdd(counts + (k == kDead ? dead_bin : (long long)k), 1);
}

// Inclusive scan of one value per thread across the block.
__device__ __forceinline__ int block_inclusive_scan(int v, int* warp_sums) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (kScanThreads / 32)) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < (kScanThreads / 32)) warp_sums[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += warp_sums[wid - 1];
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const int* __restrict__ in, long long n,
                                                              int* __restrict__ tile_sums) {
  __shared__ int ws[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q)
    if (base + q < n) s += in[base + q];
  const int inc = block_inclusive_scan(s, ws);
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = inc;
}

// Exclusive scan of the tile sums in place, one block looping over chunks.
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(int* __restrict__ sums, int ntiles) {
  __shared__ int ws[kScanThreads / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += kScanThreads) {
    const int idx = base + threadIdx.x;
    const int v = idx < ntiles ? sums[idx] : 0;
    const int inc = block_inclusive_scan(v, ws);
    const int c0 = carry;
    if (idx < ntiles) sums[idx] = c0 + inc - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = c0 + inc;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* __restrict__ in, long long n,
                                                               const int* __restrict__ tile_off,
                                                               int* __restrict__ out) {
  __shared__ int ws[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0;
    s += v[q];
  }
  const int inc = block_inclusive_scan(s, ws);
  int run = tile_off[blockIdx.x] + inc - s;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
}

__global__ void k_live_count(const int* __restrict__ offsets, long long dead_bin, int* __restrict__ n_out) {
  *n_out = offsets[dead_bin];
}

template <typename T>
__global__ void k_scatter(const Particles<T> src, const Particles<T> dst, int* __restrict__ cursor,
                          long long dead_bin) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= src.n || i >= (long long)(*src.n_dev)) return;
  const uint32_t k = src.key[i];
  if (k == kDead) return;
  const int pos = atomicAdd(cursor + k, 1);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    dst.x[q][pos] = src.x[q][i];
    dst.u[q][pos] = src.u[q][i];
  }
  dst.id[pos] = src.id[i];
  dst.key[pos] = k;
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

int scan_tiles(long long nbins) { return (int)((nbins + kScanTile - 1) / kScanTile); }

template <typename T>
void launch_sort(const Grid& g, const Particles<T>& src, const Particles<T>& dst, const SortScratch& s, int* n_out,
                 cudaStream_t stream) {
  const long long nbins = g.ncell + 1;
  const long long dead_bin = g.ncell;
  cudaMemsetAsync(s.counts, 0, sizeof(int) * nbins, stream);
  if (src.n > 0) k_hist<<<blocks_for(src.n, 256), 256, 0, stream>>>(src.key, src.n, src.n_dev, s.counts, dead_bin);
  const int ntiles = (int)((nbins + kScanTile - 1) / kScanTile);
  k_tile_sums<<<ntiles, kScanThreads, 0, stream>>>(s.counts, nbins, s.blocks);
  k_scan_tile_sums<<<1, kScanThreads, 0, stream>>>(s.blocks, ntiles);
  k_scan_apply<<<ntiles, kScanThreads, 0, stream>>>(s.counts, nbins, s.blocks, s.offsets);
  // scatter first: it reads the old count through src.n_dev, which may alias n_out.  Removed
  // particles never take a slot, so the cursor of the removed bin still holds the live count.
  if (src.n > 0) k_scatter<T><<<blocks_for(src.n, 256), 256, 0, stream>>>(src, dst, s.offsets, dead_bin);
  k_live_count<<<1, 1, 0, stream>>>(s.offsets, dead_bin, n_out);
}

template void launch_sort<float>(const Grid&, const Particles<float>&, const Particles<float>&, const SortScratch&,
                                 int*, cudaStream_t);
template void launch_sort<double>(const Grid&, const Particles<double>&, const Particles<double>&,
                                  const SortScratch&, int*, cudaStream_t);

}  // namespace grpic
