// mmc_observables_noalloc: the observables reduction of a caller-owned state
// with no device allocation by the library (declared in include/mmc.h).
//
// The reduction needs scratch for its per-block partial sums.  Here that
// scratch is a file-scope __device__ array of fixed capacity, so the entry
// point issues only kernel launches and one memset of the caller's histogram;
// it never calls cudaMalloc/cudaFree or any routine that allocates.
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/mmc.h"
#include "mmc_internal.h"

namespace {

constexpr int kNaBlock = 256;                               // threads per block
constexpr int kNaPerThread = 4;                             // cells per thread
constexpr int kNaCellsPerBlock = kNaBlock * kNaPerThread;   // 1024
constexpr int kNaMaxBlocks = 2048;
constexpr long long kNaMaxCells = (long long)kNaMaxBlocks * kNaCellsPerBlock;   // 2,097,152
constexpr int kNaSlots = 8;                                 // doubles per block

// Scratch shared by every call on a device (128 KiB; resident while the
// library stays loaded).  Host code must not use this symbol as an address.
__device__ __align__(256) double g_obs_scratch[kNaMaxBlocks * kNaSlots];

template <typename T>
__device__ __forceinline__ T warp_sum_na(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// per-block partial sums {sum mx, my, mz, |m|, |m|^2, non-finite} into part[8 b]
__global__ void __launch_bounds__(kNaBlock)
k_na_partial(const float4 *m, long long n, double *part, unsigned long long *hist, int bins, float scale) {
  __shared__ unsigned hcount[mmc::kHistMax + 1];
  __shared__ double red[kNaBlock / 32][6];
  for (int b = threadIdx.x; b <= bins; b += blockDim.x) hcount[b] = 0;
  __syncthreads();
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const long long base = (long long)blockIdx.x * kNaCellsPerBlock;
  for (int t = 0; t < kNaPerThread; ++t) {
    const long long q = base + (long long)t * kNaBlock + threadIdx.x;
    if (q >= n) break;
    const float4 v = m[q];
    if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) {
      acc[5] += 1.0;
      continue;
    }
    const double x = v.x, y = v.y, z = v.z;
    const double l2 = x * x + y * y + z * z;
    acc[0] += x; acc[1] += y; acc[2] += z;
    acc[3] += sqrt(l2);
    acc[4] += l2;
    // same FP32 bin decision as the context's observables
    const float r2 = __fmaf_rn(v.z, v.z, __fmaf_rn(v.y, v.y, __fmul_rn(v.x, v.x)));
    const float tb = __fmul_rn(__fsqrt_rn(r2), scale);
    const int b = tb >= (float)bins ? bins : (int)tb;
    atomicAdd(&hcount[b], 1u);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double w = warp_sum_na(acc[k]);
    if (lane == 0) red[warp][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0;
    for (int w = 0; w < kNaBlock / 32; ++w) s += red[w][threadIdx.x];
    part[(long long)kNaSlots * blockIdx.x + threadIdx.x] = s;
  }
  for (int b = threadIdx.x; b <= bins; b += blockDim.x)
    if (hcount[b]) atomicAdd(&hist[b], (unsigned long long)hcount[b]);
}

// fixed-order sum of the partials; out = {<mx>, <my>, <mz>, <|m|>, <|m|^2>, non-finite, n valid, 0}
__global__ void k_na_final(const double *part, int nblocks, long long n, double *out) {
  __shared__ double red[6][32];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 6; ++k) acc[k] += part[(long long)kNaSlots * b + k];
  for (int k = 0; k < 6; ++k) {
    const double w = warp_sum_na(acc[k]);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[6];
    for (int k = 0; k < 6; ++k) {
      tot[k] = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot[k] += red[k][w];
    }
    const double nvalid = (double)n - tot[5];
    const double d = nvalid > 0 ? nvalid : 1.0;
    for (int k = 0; k < 5; ++k) out[k] = tot[k] / d;
    out[5] = tot[5];
    out[6] = nvalid;
    out[7] = 0.0;
  }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

mmc_status na_fail(mmc_status s, const std::string &msg) {
  mmc::set_last_error(msg.c_str());
  return s;
}

}  // namespace

extern "C" mmc_status mmc_observables_noalloc(const float *m, int64_t n, int hist_bins, double hist_max,
                                              double *out, unsigned long long *hist, void *cuda_stream) {
  if (!m || !out || !hist) return na_fail(MMC_ERR_ARG, "null pointer");
  if (n < 1) return na_fail(MMC_ERR_ARG, "n must be >= 1");
  if (n > kNaMaxCells) return na_fail(MMC_ERR_ARG, "n exceeds the built-in scratch capacity of 2097152 cells");
  if (hist_bins < 1 || hist_bins > mmc::kHistMax) return na_fail(MMC_ERR_ARG, "hist_bins must be in [1, 1024]");
  if (!(hist_max > 0)) return na_fail(MMC_ERR_ARG, "hist_max must be > 0");
  // m is read as float4 and out / hist written as 8-byte words: a misaligned
  // pointer would fault the kernel, so it is rejected before any launch
  if ((reinterpret_cast<uintptr_t>(m) & 15u) != 0) return na_fail(MMC_ERR_ARG, "m must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(out) & 7u) != 0 || (reinterpret_cast<uintptr_t>(hist) & 7u) != 0)
    return na_fail(MMC_ERR_ARG, "out and hist must be 8-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(MMC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(MMC_ERR_UNSUPPORTED, "device index above 63");
  if (cuda_stream) {
    // the scratch address below is the current device's; a stream of another
    // device would run the kernels against the wrong device's memory
    int sdev = -1;
    e = cudaStreamGetDevice((cudaStream_t)cuda_stream, &sdev);
    if (e != cudaSuccess) return na_fail(MMC_ERR_ARG, std::string("cudaStreamGetDevice: ") + cudaGetErrorString(e));
    if (sdev != dev) return na_fail(MMC_ERR_ARG, "cuda_stream belongs to another device than the current one");
  }
  double *scratch = nullptr;
  {
    // once per device, with that device current: the scratch's device address
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_obs_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(MMC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  e = cudaMemsetAsync(hist, 0, (size_t)(hist_bins + 1) * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return na_fail(MMC_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const int nblocks = (int)((n + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
  const float scale = (float)hist_bins / (float)hist_max;
  k_na_partial<<<nblocks, kNaBlock, 0, st>>>(reinterpret_cast<const float4 *>(m), n, scratch, hist, hist_bins,
                                              scale);
  k_na_final<<<1, 256, 0, st>>>(scratch, nblocks, n, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(MMC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return MMC_OK;
}
