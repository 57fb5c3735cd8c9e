// Arguments of the demag convolution kernels (Sec. III, Eq. 14) and the load of
// M = Ms0 m from the split sublattice layout, shared by the generic kernels
// (k_demag.cu) and the interleaved 2D kernels (k_demag_il.cuh).
#pragma once

#include "fft.cuh"
#include "mmc_internal.h"

namespace mmc {

template <typename R>
struct DemagArgs {
  using C = typename Cx<R>::T;
  const ChainDev *chains;
  const int *blk_chain;
  const long long *blk_first;
  const float4 *m;
  const float4 *tab;
  const float *ms;
  const float *ms_lo;   // per-cell Ms0 minus its FP32 value (FP64 and float-float convolutions)
  C *S;
  const R *const *nhat;
  const C *tw;
  float4 *heff;
  double *Hd;
  int Hd_chain;
  const R *m_nat;     // optional natural-order input (3 per cell) instead of the split state
  R Ms_override;      // > 0: uniform Ms0 used with m_nat
  MmcCheck *ck;       // checked builds: the record (checked.cuh)
  int nchains;        // entries of the chain table
};

// the block's chain, checked against the chain table
template <typename R>
__device__ __forceinline__ int demag_chain_of_block(const DemagArgs<R> &A) {
  return (int)MMC_CK(A.ck, A.blk_chain[blockIdx.x], 0, A.nchains, kCkDemagBlock);
}

// elements of a chain's spectrum region (rows rounded up to four in 2D)
__device__ __forceinline__ long long spectrum_elems(const ChainDev &ch) {
  const long long rows = ch.Pz == 1 ? ((ch.nrows + 3) & ~3) : ch.nrows;
  return 3 * rows * ch.Sx;
}

__device__ __forceinline__ int pairs_per_block(int Px) {
  const int G = Px >= 8 ? Px >> 3 : 1;
  int np = (int)blockDim.x / (3 * G);
  return np < 1 ? 1 : (np > 8 ? 8 : np);
}

// M = Ms0 m of cell (x, row r) from the split layout, formed in the convolution's precision
template <typename R>
__device__ __forceinline__ void load_M(const ChainDev &ch, const float4 *m, const float *ms, const float *ms_lo,
                                       int r, int x, R &Mx, R &My, R &Mz, MmcCheck *ck = nullptr) {
  const int k = (int)divq((unsigned)r, ch.ny_m, ch.ny_l), j = r - k * ch.ny;
  const int col = (x + j + k) & 1;
  const long long S = (long long)ch.nrows * ch.hx;
  const long long idx = MMC_CK(ck, (long long)col * S + (long long)r * ch.hx + (x >> 1), 0, 2 * S, kCkDemagM);
  const float4 v = m[ch.m_off + idx];
  R Ms = ch.ms_off >= 0 ? (R)ms[ch.ms_off + idx] : (R)ch.Ms0d;
  // the wider formats take per-cell Ms0 as the pair (FP32 value, rest)
  if constexpr (sizeof(R) == 8)
    if (ch.ms_off >= 0 && ms_lo) Ms = Ms + (R)ms_lo[ch.ms_off + idx];
  Mx = Ms * (R)v.x;
  My = Ms * (R)v.y;
  Mz = Ms * (R)v.z;
}

}  // namespace mmc
