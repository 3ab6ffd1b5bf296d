// Particle removal and counting sort by cell (not in the paper: the paper names no boundary
// treatment; removed particles carry key kDead and are dropped here).
//
//   1. histogram of the keys into ncell + 1 bins (the last bin collects removed particles);
//   2. exclusive prefix sum of the bins (block-level warp-shuffle scans, three passes);
//   3. scatter of x, u, id, key into the alternate buffers at bin offset + running count.
// The live count (start of the removed bin) is left in device memory, so no host round
// trip is needed between steps.  Within a cell the order is not stable.
#include <algorithm>

#include "common.cuh"

namespace grpic {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Runs of equal keys in a warp.  Sorted or nearly sorted keys (the store is cell-sorted and particles
// move less than a cell per step) put equal keys in adjacent lanes; each maximal run of equal keys
// among the warp's valid lanes (a prefix of the warp) shares one atomic, taken by its first lane.
// Equal keys in runs that are not adjacent simply take one atomic each.  The run's first lane and
// its length come from one shuffle and two ballots (all 32 lanes call it).
struct KeyRun {
  bool head;  // this lane starts a run
  int first;  // lane that starts this lane's run
  int len;    // length of the run (meaningful on its first lane)
};
__device__ __forceinline__ KeyRun key_run(bool valid, uint32_t k) {
  const int lane = threadIdx.x & 31;
  const unsigned vmask = __ballot_sync(0xffffffffu, valid);
  const uint32_t prev = __shfl_up_sync(0xffffffffu, k, 1);
  KeyRun r;
  r.head = valid && (lane == 0 || prev != k);
  const unsigned heads = __ballot_sync(0xffffffffu, r.head);
  const unsigned upto = heads & (0xffffffffu >> (31 - lane));  // heads at or below this lane
  r.first = upto ? 31 - __clz(upto) : 0;
  const unsigned above = lane == 31 ? 0u : heads & (0xffffffffu << (lane + 1));  // heads above this lane
  const int next = above ? __ffs(above) - 1 : 32;
  r.len = min(next, __popc(vmask)) - lane;
  return r;
}

__global__ void k_hist(const uint32_t* __restrict__ key, long long n, const int* __restrict__ n_dev,
                       int* __restrict__ counts, long long dead_bin) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool valid = i < n && i < (long long)(*n_dev);
  const uint32_t k = valid ? key[i] : kDead;
  const KeyRun r = key_run(valid, k);
  if (r.head) atomicAdd(counts + (k == kDead ? dead_bin : (long long)k), r.len);
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

// Each thread moves kScatterItems records, from kScatterItems consecutive blocks' worth of the store
// (chunk j of block b covers [(b * items + j) * blockDim, ...)), so a warp's lanes stay contiguous.
// Every record and key is read before any slot is known, so that the record loads and the atomics
// are in flight together (k_scatter at 96^3: 145 -> 122 us).  Two items per thread measured the
// same as one.
constexpr int kScatterItems = 1;

template <typename T>
__global__ void k_scatter(const Particles<T> src, const Particles<T> dst, int* __restrict__ cursor,
                          long long dead_bin) {
  const long long live_n = min(src.n, (long long)(*src.n_dev));
  uint32_t k[kScatterItems], idv[kScatterItems];
  T xv[kScatterItems][4], uv[kScatterItems][4];
  bool in_range[kScatterItems];
#pragma unroll
  for (int j = 0; j < kScatterItems; ++j) {
    const long long i = ((long long)blockIdx.x * kScatterItems + j) * blockDim.x + threadIdx.x;
    in_range[j] = i < live_n;
    k[j] = in_range[j] ? src.key[i] : kDead;
    idv[j] = 0;
    if (in_range[j] && k[j] != kDead) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xv[j][q] = src.x[q][i];
        uv[j][q] = src.u[q][i];
      }
      idv[j] = src.id[i];
    }
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kScatterItems; ++j) {
    // one atomic per run of lanes with the same cell, each lane at its rank in the run; removed
    // particles form runs of their own and take no slot
    const KeyRun r = key_run(in_range[j], k[j]);
    int first = 0;
    if (r.head && k[j] != kDead) first = atomicAdd(cursor + k[j], r.len);
    const int pos = __shfl_sync(0xffffffffu, first, r.first) + (lane - r.first);
    if (in_range[j] && k[j] != kDead) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        dst.x[q][pos] = xv[j][q];
        dst.u[q][pos] = uv[j][q];
      }
      dst.id[pos] = idv[j];
      dst.key[pos] = k[j];
    }
  }
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---- batched: all (instance, species) pairs share one bin array -------------------------------
template <typename T>
__global__ void k_batch_hist(const InstDesc<T>* __restrict__ desc, const BlockEntry* __restrict__ blk, int nblk,
                             int* __restrict__ counts) {
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    const BlockEntry e = blk[bi];
    const InstDesc<T>& D = desc[e.inst >> 2];
    const SpeciesDesc<T>& S = D.sp[e.inst & 3];
    const Particles<T>& P = S.buf[*S.cur];
    const long long i = (long long)e.block * blockDim.x + threadIdx.x;
    const bool valid = i < P.n && i < (long long)(*P.n_dev);
    const uint32_t k = valid ? P.key[i] : kDead;
    const KeyRun r = key_run(valid, k);  // the block belongs to one (instance, species): warp-uniform
    if (r.head) atomicAdd(counts + S.bin_base + (k == kDead ? D.g.ncell : (long long)k), r.len);
  }
}

template <typename T>
__global__ void k_batch_base(const InstDesc<T>* __restrict__ desc, const int* __restrict__ pairs, int npairs,
                             const int* __restrict__ offsets, int* __restrict__ base) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const InstDesc<T>& D = desc[pairs[p] >> 2];
  base[p] = offsets[D.sp[pairs[p] & 3].bin_base];
}

template <typename T>
__global__ void k_batch_scatter(const InstDesc<T>* __restrict__ desc, const BlockEntry* __restrict__ blk, int nblk,
                                const int* __restrict__ pair_of_inst, const int* __restrict__ base,
                                int* __restrict__ cursor) {
  for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x) {
    const BlockEntry e = blk[bi];
    const InstDesc<T>& D = desc[e.inst >> 2];
    const SpeciesDesc<T>& S = D.sp[e.inst & 3];
    const int cur = *S.cur;
    const Particles<T>& src = S.buf[cur];
    const Particles<T>& dst = S.buf[1 - cur];
    const long long i = (long long)e.block * blockDim.x + threadIdx.x;
    const bool in_range = i < src.n && i < (long long)(*src.n_dev);
    const uint32_t k = in_range ? src.key[i] : kDead;
    const bool live = in_range && k != kDead;
    T xv[4], uv[4];
    uint32_t idv = 0;
    if (live) {  // read ahead of the atomic, as in k_scatter
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xv[q] = src.x[q][i];
        uv[q] = src.u[q][i];
      }
      idv = src.id[i];
    }
    const KeyRun r = key_run(in_range, k);
    const int lane = threadIdx.x & 31;
    int first = 0;
    if (r.head && k != kDead) first = atomicAdd(cursor + S.bin_base + k, r.len);
    const int run0 = __shfl_sync(0xffffffffu, first, r.first);  // every lane takes part
    if (!live) continue;
    const int pos = run0 + (lane - r.first) - base[pair_of_inst[e.inst]];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dst.x[q][pos] = xv[q];
      dst.u[q][pos] = uv[q];
    }
    dst.id[pos] = idv;
    dst.key[pos] = k;
  }
}

// live count and buffer flip of every pair (after the scatter has read the old index)
template <typename T>
__global__ void k_batch_finish(const InstDesc<T>* __restrict__ desc, const int* __restrict__ pairs, int npairs,
                               const int* __restrict__ offsets, const int* __restrict__ base) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const InstDesc<T>& D = desc[pairs[p] >> 2];
  const SpeciesDesc<T>& S = D.sp[pairs[p] & 3];
  const int cur = *S.cur;
  *const_cast<int*>(S.buf[cur].n_dev) = offsets[S.bin_base + D.g.ncell] - base[p];  // shared by both buffers
  *S.cur = 1 - cur;
}

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
  if (src.n > 0)
    k_scatter<T><<<blocks_for(src.n, 256 * kScatterItems), 256, 0, stream>>>(src, dst, s.offsets, dead_bin);
  k_live_count<<<1, 1, 0, stream>>>(s.offsets, dead_bin, n_out);
}

// pair_of_inst: for each (instance * 4 + species) the index of its pair (stored after `base`).
template <typename T>
void launch_batch_sort(const BatchTables<T>& bt, cudaStream_t stream) {
  if (bt.npairs == 0) return;
  cudaMemsetAsync(bt.counts, 0, sizeof(int) * bt.nbins, stream);
  const unsigned nb = (unsigned)std::min(bt.npart, bt.persist_blocks);
  const int* pair_of_inst = bt.pair_base + bt.npairs;
  if (bt.npart > 0) k_batch_hist<T><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart, bt.counts);
  const int ntiles = (int)((bt.nbins + kScanTile - 1) / kScanTile);
  k_tile_sums<<<ntiles, kScanThreads, 0, stream>>>(bt.counts, bt.nbins, bt.tiles);
  k_scan_tile_sums<<<1, kScanThreads, 0, stream>>>(bt.tiles, ntiles);
  k_scan_apply<<<ntiles, kScanThreads, 0, stream>>>(bt.counts, bt.nbins, bt.tiles, bt.offsets);
  k_batch_base<T><<<blocks_for(bt.npairs, 128), 128, 0, stream>>>(bt.desc, bt.pairs, bt.npairs, bt.offsets,
                                                                     bt.pair_base);
  if (bt.npart > 0)
    k_batch_scatter<T><<<nb, 128, 0, stream>>>(bt.desc, bt.part, bt.npart, pair_of_inst, bt.pair_base, bt.offsets);
  k_batch_finish<T><<<blocks_for(bt.npairs, 128), 128, 0, stream>>>(bt.desc, bt.pairs, bt.npairs, bt.offsets,
                                                                       bt.pair_base);
}

template void launch_batch_sort<float>(const BatchTables<float>&, cudaStream_t);
template void launch_batch_sort<double>(const BatchTables<double>&, cudaStream_t);

template void launch_sort<float>(const Grid&, const Particles<float>&, const Particles<float>&, const SortScratch&,
                                 int*, cudaStream_t);
template void launch_sort<double>(const Grid&, const Particles<double>&, const Particles<double>&,
                                  const SortScratch&, int*, cudaStream_t);

}  // namespace grpic
