// Angular-deviation histogram of one chain (Sec. II, Fig. 1d-f): the polar
// angle of every cell to the configuration's mean direction, counted in equal
// bins on [lo, hi) (angles outside go to the last entry).  FP64 angles of the
// FP32 state, so the bin decisions equal those of an FP64 evaluation.
#include "angles.h"

namespace mmc {

constexpr int kAngBlock = 256;

__global__ void k_angle_hist(const ChainDev *chains, int c, const float4 *m, double n0, double n1, double n2,
                             double lo, double scale, int bins, unsigned long long *hist) {
  extern __shared__ unsigned int sh[];
  for (int b = threadIdx.x; b <= bins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const ChainDev &ch = chains[c];
  const long long S = (long long)ch.nrows * ch.hx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * S; t += (long long)gridDim.x * blockDim.x) {
    const int color = t >= S ? 1 : 0;
    const long long q = t - color * S;
    const int row = (int)(q / ch.hx), s = (int)(q - (long long)row * ch.hx);
    const int k = row / ch.ny, j = row - k * ch.ny;
    const int i = 2 * s + ((j + k + color) & 1);
    if (i >= ch.nx) continue;
    const float4 v = m[ch.m_off + t];
    const double x = v.x, y = v.y, z = v.z;
    const double l = sqrt(x * x + y * y + z * z);
    double ct = l > 0 ? (x * n0 + y * n1 + z * n2) / l : 1.0;
    ct = fmin(1.0, fmax(-1.0, ct));
    const double f = (acos(ct) - lo) * scale;
    const int b = (f >= 0.0 && f < (double)bins) ? (int)f : bins;
    atomicAdd(&sh[b], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b <= bins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

void launch_angle_hist(const Launch &L, const ChainDev *chains, int c, long long slots, const float4 *m,
                       const double n[3], double lo, double hi, int bins, unsigned long long *hist) {
  long long nb = (2 * slots + kAngBlock - 1) / kAngBlock;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  const double scale = (double)bins / (hi - lo);
  k_angle_hist<<<(int)nb, kAngBlock, (size_t)(bins + 1) * sizeof(unsigned int), L.stream>>>(
      chains, c, m, n[0], n[1], n[2], lo, scale, bins, hist);
  ++*L.counter;
}

}  // namespace mmc
