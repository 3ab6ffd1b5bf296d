// Sustained FMA rate of the CUDA cores (roofline denominator of the ALU-bound push): every
// lane runs 8 independent fused-multiply-add chains; the result is stored so nothing is dead.
#include <cuda_runtime.h>

#include "../../include/grpic.h"
#include "metric.cuh"
#include "push_core.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  T v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = (T)(threadIdx.x + q) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = fma(v[q], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 8; ++q) s += v[q];
  if (s == T(12345.678)) out[0] = s;  // practically never true; keeps the chains live
}

template <typename T>
double measure(int iters) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return -1.0;
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess) return -1.0;
  const double flops = 2.0 * 8.0 * 16.0 * (double)iters * (double)blocks * threads;
  return flops / (best * 1e-3);
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014) as a counter-based uniform generator.
__device__ __forceinline__ double uniform01(unsigned long long k) {
  unsigned long long z = k + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// Relative deviation of SeededOps64 from the IEEE operations over log-uniform arguments in
// [1e-8, 1e8]; maxima by atomicMax on the bit patterns (non-negative doubles order as integers).
__global__ void k_check_newton64(long long n, unsigned long long* worst) {
  double e_rcp = 0.0, e_div = 0.0, e_root = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = exp10(-8.0 + 16.0 * uniform01(2 * i));
    const double y = exp10(-8.0 + 16.0 * uniform01(2 * i + 1));
    const double r_ieee = 1.0 / x, q_ieee = y / x, s_ieee = sqrt(x);
    e_rcp = fmax(e_rcp, fabs(grpic::SeededOps64::rcp(x) - r_ieee) / r_ieee);
    e_div = fmax(e_div, fabs(grpic::SeededOps64::div(y, x) - q_ieee) / q_ieee);
    e_root = fmax(e_root, fabs(grpic::SeededOps64::root(x) - s_ieee) / s_ieee);
  }
  atomicMax(worst + 0, (unsigned long long)__double_as_longlong(e_rcp));
  atomicMax(worst + 1, (unsigned long long)__double_as_longlong(e_div));
  atomicMax(worst + 2, (unsigned long long)__double_as_longlong(e_root));
}

// widen / narrow of the push against the hardware conversions, bit for bit: float bit
// patterns with a normal or infinite/NaN exponent, and doubles whose exponent lies in or just
// around the binary32 normal range, a quarter of them exact rounding ties.
__global__ void k_check_conversions(long long n, unsigned long long* bad) {
  unsigned long long nb_w = 0, nb_n = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long r = (unsigned long long)(uniform01(3 * i) * 0x1.0p53);
    const unsigned fu = (unsigned)(r & 0xffffffffull);
    if (((fu >> 23) & 0xffu) != 0u) {
      const float f = __uint_as_float(fu);
      const double w = grpic::widen(f), h = (double)f;
      const bool same = (f != f) ? (w != w) : (__double_as_longlong(w) == __double_as_longlong(h));
      nb_w += same ? 0 : 1;
    }
    const unsigned long long r2 = (unsigned long long)(uniform01(3 * i + 1) * 0x1.0p53);
    const unsigned e = 893u + (unsigned)(uniform01(3 * i + 2) * 262.0);  // 893 .. 1154
    unsigned long long bits = ((r2 & 1ull) << 63) | ((unsigned long long)e << 52) | ((r2 >> 1) & 0xfffffffffffffull);
    if ((i & 3) == 0) bits = (bits & ~0x1fffffffull) | 0x10000000ull;  // a tie
    const double d = __longlong_as_double((long long)bits);
    nb_n += (__float_as_uint(grpic::narrow(d)) == __float_as_uint(__double2float_rn(d))) ? 0 : 1;
  }
  if (nb_w) atomicAdd(bad + 0, nb_w);
  if (nb_n) atomicAdd(bad + 1, nb_n);
}

}  // namespace

extern "C" grpic_status grpic_check_conversions(int64_t n, int64_t mismatches[2]) {
  if (n <= 0 || !mismatches) return GRPIC_ERR_INVALID;
  unsigned long long* w = nullptr;
  if (cudaMalloc(&w, 2 * sizeof(unsigned long long)) != cudaSuccess) return GRPIC_ERR_OOM;
  cudaMemset(w, 0, 2 * sizeof(unsigned long long));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_check_conversions<<<sms * 4, 256>>>(n, w);
  unsigned long long h[2] = {0, 0};
  const cudaError_t e = cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(w);
  if (e != cudaSuccess) return GRPIC_ERR_CUDA;
  mismatches[0] = (int64_t)h[0];
  mismatches[1] = (int64_t)h[1];
  return GRPIC_OK;
}

extern "C" grpic_status grpic_check_newton64(int64_t n, double max_rel[3]) {
  if (n <= 0 || !max_rel) return GRPIC_ERR_INVALID;
  unsigned long long* w = nullptr;
  if (cudaMalloc(&w, 3 * sizeof(unsigned long long)) != cudaSuccess) return GRPIC_ERR_OOM;
  cudaMemset(w, 0, 3 * sizeof(unsigned long long));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_check_newton64<<<sms * 4, 256>>>(n, w);
  unsigned long long h[3] = {0, 0, 0};
  const cudaError_t e = cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(w);
  if (e != cudaSuccess) return GRPIC_ERR_CUDA;
  for (int q = 0; q < 3; ++q) max_rel[q] = __builtin_bit_cast(double, h[q]);
  return GRPIC_OK;
}

extern "C" grpic_status grpic_probe_fma_peak(int precision, double* flops_per_s) {
  if (!flops_per_s) return GRPIC_ERR_INVALID;
  double v;
  if (precision == GRPIC_FP32_MIXED)
    v = measure<float>(4096);
  else if (precision == GRPIC_FP64)
    v = measure<double>(64);
  else
    return GRPIC_ERR_INVALID;
  if (!(v > 0.0)) return GRPIC_ERR_CUDA;
  *flops_per_s = v;
  return GRPIC_OK;
}
