// Bounds-checked builds of the sweep and demag kernels (compiled with
// -DMMC_CHECKED; compute-sanitizer is not available everywhere this runs).
//
// Every global-memory index those kernels compute is compared, before the
// access, with the range of the buffer region it belongs to (a chain's colour of
// m, its h_eff, its per-cell tables, its spectrum, a tensor set, a block table).
// An index outside its range is counted, the first one is recorded with its
// range and the access site in a device word, and the access goes to the first
// element of the range instead: a wrong index is reported by
// mmc_check_report, it never faults.  Bulk asynchronous copies are checked on
// their first and last source element.  In normal builds MMC_CK(...) is the
// index itself and nothing is added.
#pragma once

#include <cuda_runtime.h>

namespace mmc {

struct MmcCheck {
  unsigned long long count;     // indices found out of range
  long long index, lo, hi;      // the first of them and the range [lo, hi) it had to lie in
  int site;                     // where (MmcCheckSite)
  int pad;
};

// access sites (reported by mmc_check_report; names in check_site_name)
enum MmcCheckSite : int {
  kCkSweepBlock = 1,            // sweep block table entry
  kCkSweepCell,                 // the updated cell (load and store)
  kCkSweepNeighbour,            // a neighbour in the other colour
  kCkSweepField,                // h_eff of the cell
  kCkSweepTable,                // per-cell material tables
  kCkSweepDebug,                // decision / accept outputs of the debug pass
  kCkBandItem,                  // banded pass: work item
  kCkBandCopy,                  // banded pass: bulk-copy source rows
  kCkDemagM,                    // demag: m (and per-cell Ms0) read by the forward rows
  kCkDemagSpectrum,             // demag: spectrum element or tile
  kCkDemagTensor,               // demag: tensor spectrum
  kCkDemagField,                // demag: h_eff / H_d written by the inverse rows
  kCkDemagBlock,                // demag block table entry
  kCkFusedCopy,                 // fused kernels: bulk-copy source rows
  kCkFusedState,                // fused kernels: m written by the pass
  kCkSiteCount
};

#ifdef MMC_CHECKED
constexpr bool kChecked = true;

// record a bad index and give back a valid one (lo when the range is not empty)
__host__ __device__ inline long long ck_fail(MmcCheck *ck, long long i, long long lo, long long hi, int site) {
  if (ck) {
#ifdef __CUDA_ARCH__
    const unsigned long long n = atomicAdd(&ck->count, 1ull);
#else
    const unsigned long long n = ck->count++;
#endif
    if (n == 0ull) {
      ck->index = i;
      ck->lo = lo;
      ck->hi = hi;
      ck->site = site;
    }
  }
  return lo < hi ? lo : 0;
}

// (a launch without a record, ck == nullptr, is not checked)
__host__ __device__ __forceinline__ long long ck_index(MmcCheck *ck, long long i, long long lo, long long hi,
                                                       int site) {
  return (!ck || (i >= lo && i < hi)) ? i : ck_fail(ck, i, lo, hi, site);
}

// [i, i + n) inside [lo, hi): gives back i, or lo after recording i
__host__ __device__ __forceinline__ long long ck_range(MmcCheck *ck, long long i, long long n, long long lo,
                                                       long long hi, int site) {
  return (!ck || (i >= lo && i + n <= hi)) ? i : ck_fail(ck, i, lo, hi, site);
}

#define MMC_CK(ck, i, lo, hi, site) ::mmc::ck_index((ck), (long long)(i), (long long)(lo), (long long)(hi), (site))
#define MMC_CKR(ck, i, n, lo, hi, site) \
  ::mmc::ck_range((ck), (long long)(i), (long long)(n), (long long)(lo), (long long)(hi), (site))
#else
constexpr bool kChecked = false;
#define MMC_CK(ck, i, lo, hi, site) (i)
#define MMC_CKR(ck, i, n, lo, hi, site) (i)
#endif

}  // namespace mmc
