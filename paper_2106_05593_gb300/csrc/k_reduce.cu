// Reductions and state movement:
//  - observables (Sec. II, Figs. 1-2): <m>, <|m|>, <|m|^2> accumulated in FP64,
//    |m| histogram with integer counters, non-finite count;
//  - energy terms (Eqs. 7, 10-12, 14, 15) in FP64 per cell, reduced in a fixed
//    order (per-block partials, then one block per chain);
//  - natural-order <-> checkerboard-split copies and the random initial state.
#include <cmath>

#include "mmc_internal.h"
#include "philox.cuh"

namespace mmc {

__device__ __forceinline__ bool slot_cell(const ChainDev &ch, long long q2, int &color, long long &q,
                                          int &i, int &row) {
  const long long S = (long long)ch.nrows * ch.hx;
  color = q2 >= S ? 1 : 0;
  q = q2 - (long long)color * S;
  row = (int)(q / ch.hx);
  const int s = (int)(q - (long long)row * ch.hx);
  const int j = row % ch.ny, k = row / ch.ny;
  i = 2 * s + ((j + k + color) & 1);
  return i < ch.nx;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// observables: partial sums per block
__global__ void __launch_bounds__(kReduceBlock)
k_obs_partial(const ChainDev *chains, const int *blk_chain, const long long *blk_first,
              const float4 *m, double *part, unsigned long long *hist, int bins, float scale) {
  pdl_enter();
  __shared__ unsigned hcount[kHistMax + 1];
  __shared__ double red[kReduceBlock / 32][6];
  const int c = blk_chain[blockIdx.x];
  const ChainDev &ch = chains[c];
  for (int b = threadIdx.x; b <= bins; b += blockDim.x) hcount[b] = 0;
  __syncthreads();
  const long long S2 = 2LL * ch.nrows * ch.hx;
  const long long base = (long long)(blockIdx.x - blk_first[c]) * kReduceBlock * 4;
  double sx = 0, sy = 0, sz = 0, sl = 0, sl2 = 0, nf = 0;
  for (int t = 0; t < 4; ++t) {
    const long long q2 = base + t * kReduceBlock + threadIdx.x;
    if (q2 >= S2) break;
    int color, i, row;
    long long q;
    if (!slot_cell(ch, q2, color, q, i, row)) continue;
    const float4 v = m[ch.m_off + q2];
    if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) { nf += 1; continue; }
    const double x = v.x, y = v.y, z = v.z;
    const double l2 = x * x + y * y + z * z;
    sx += x; sy += y; sz += z;
    sl += sqrt(l2);
    sl2 += l2;
    // FP32 bin decision: r = sqrt(fma(z,z,fma(y,y,x*x))), bin = (int)(r * bins/hmax)
    const float r2 = __fmaf_rn(v.z, v.z, __fmaf_rn(v.y, v.y, __fmul_rn(v.x, v.x)));
    const float tb = __fmul_rn(__fsqrt_rn(r2), scale);
    const int b = tb >= (float)bins ? bins : (int)tb;
    atomicAdd(&hcount[b], 1u);
  }
  double vals[6] = {sx, sy, sz, sl, sl2, nf};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double w = warp_sum(vals[k]);
    if (lane == 0) red[warp][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double acc = 0;
    for (int w = 0; w < kReduceBlock / 32; ++w) acc += red[w][threadIdx.x];
    part[8LL * blockIdx.x + threadIdx.x] = acc;
  }
  unsigned long long *hc = hist + (long long)c * (bins + 1);
  for (int b = threadIdx.x; b <= bins; b += blockDim.x)
    if (hcount[b]) atomicAdd(&hc[b], (unsigned long long)hcount[b]);
}

// one block per chain: fixed-order sum of the chain's partials
__global__ void k_obs_final(const ChainDev *chains, ChainState *st, const long long *blk_first,
                            const double *part, double *out, int accumulate) {
  pdl_enter();
  __shared__ double red[6][32];
  const int c = blockIdx.x;
  const long long b0 = blk_first[c], b1 = blk_first[c + 1];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long b = b0 + threadIdx.x; b < b1; b += blockDim.x)
    for (int k = 0; k < 6; ++k) acc[k] += part[8 * b + k];
  for (int k = 0; k < 6; ++k) {
    const double w = warp_sum(acc[k]);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[6];
    for (int k = 0; k < 6; ++k) {
      tot[k] = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot[k] += red[k][w];
    }
    const double nvalid = (double)chains[c].ncell - tot[5];
    if (accumulate) {
      ChainState &s = st[c];
      s.sum_m[0] += tot[0]; s.sum_m[1] += tot[1]; s.sum_m[2] += tot[2];
      s.sum_len += tot[3]; s.sum_len2 += tot[4];
      s.nsamples += (unsigned long long)nvalid;
      s.nsnap += 1;
      s.nonfinite += (unsigned long long)tot[5];
    } else {
      double *o = out + 8LL * c;
      for (int k = 0; k < 6; ++k) o[k] = tot[k];
      o[6] = nvalid;
    }
  }
}

void launch_obs(const Launch &L, const ObsLaunch &P) {
  launch_pdl(k_obs_partial, P.nblocks, kReduceBlock, 0, L.stream, P.chains, P.blk_chain, P.blk_first, P.m,
                                                           P.part, P.hist, P.bins, P.scale);
  launch_pdl(k_obs_final, P.nchains, 128, 0, L.stream, P.chains, P.st, P.blk_first, P.part, P.out,
                                                P.accumulate);
  *L.counter += 2;
}

// ---------------------------------------------------------------------------
// energy of one chain, FP64 per cell
__global__ void __launch_bounds__(kReduceBlock)
k_energy_partial(const ChainDev *chains, int c, const float4 *m, const double *etab,
                 const double *Hd, EnergyCoef E, double *part) {
  __shared__ double red[kReduceBlock / 32][6];
  const ChainDev &ch = chains[c];
  const long long S = (long long)ch.nrows * ch.hx;
  const long long S2 = 2 * S;
  double ex = 0, dm = 0, an = 0, ze = 0, lo = 0, de = 0;
  for (int t = 0; t < 4; ++t) {
    const long long q2 = (long long)blockIdx.x * kReduceBlock * 4 + t * kReduceBlock + threadIdx.x;
    if (q2 >= S2) break;
    int color, i, row;
    long long q;
    if (!slot_cell(ch, q2, color, q, i, row)) continue;
    const int j = row % ch.ny, k = row / ch.ny;
    const float4 v = m[ch.m_off + q2];
    const double x = v.x, y = v.y, z = v.z;
    const long long nat = i + (long long)ch.nx * row;
    // bonds to the + neighbours (each bond once)
    const float4 *mo = m + ch.m_off + (long long)(1 - color) * S;
    const int p = (j + k + color) & 1;
    const int s = (int)(q - (long long)row * ch.hx);
    for (int a = 0; a < 3; ++a) {
      int ii = i, jj = j, kk = k;
      if (a == 0) { ii = i + 1; if (ii >= ch.nx) { if (!(ch.pbc & 1)) continue; ii = 0; } }
      if (a == 1) { jj = j + 1; if (jj >= ch.ny) { if (!(ch.pbc & 2)) continue; jj = 0; } }
      if (a == 2) { kk = k + 1; if (kk >= ch.nz) { if (!(ch.pbc & 4)) continue; kk = 0; } }
      float4 u;
      if (a == 0) u = mo[(long long)row * ch.hx + ((ii - 1 + p) >> 1)];
      else u = mo[(long long)(jj + ch.ny * kk) * ch.hx + s];
      double sc = 1.0;
      if ((ch.flags & F_GRAIN) && u.w != v.w) sc = ch.gscale;
      const double dx = x - u.x, dy = y - u.y, dz = z - u.z;
      ex += sc * E.cex[a] * (dx * dx + dy * dy + dz * dz);
      if (a < 2 && (ch.flags & F_DMI)) {
        // -(V D0 / h_a) (m_q,z m_r,a - m_q,a m_r,z)
        const double ua = a == 0 ? (double)u.x : (double)u.y;
        const double qa = a == 0 ? x : y;
        dm += -sc * E.cdmi[a] * (z * ua - qa * (double)u.z);
      }
    }
    const double l2 = x * x + y * y + z * z;
    const double len = sqrt(l2);
    double c2, c4, me2, Ms, K1, K2, e0, e1, e2;
    if (etab) {
      const double *et = etab + 10 * nat;
      c2 = et[0]; c4 = et[1]; me2 = et[2]; Ms = et[3]; K1 = et[4]; K2 = et[5];
      e0 = et[6]; e1 = et[7]; e2 = et[8];
    } else {
      c2 = E.c2; c4 = E.c4; me2 = E.me2; Ms = E.Ms0; K1 = E.K1T; K2 = E.K2T;
      e0 = E.e[0]; e1 = E.e[1]; e2 = E.e[2];
    }
    const double dq = l2 - me2;
    lo += c2 * l2 + c4 * dq * dq;
    if (len > 0) {
      const double ux = x / len, uy = y / len, uz = z / len;
      if (E.cubic) {
        const double a2 = ux * ux, b2 = uy * uy, g2 = uz * uz;
        an += E.V * (K1 * (a2 * b2 + a2 * g2 + b2 * g2) + K2 * a2 * b2 * g2);
      } else {
        const double d = ux * e0 + uy * e1 + uz * e2;
        const double sn = 1.0 - d * d;
        an += E.V * (K1 * sn + K2 * sn * sn);
      }
    }
    ze += -E.V * Ms * (x * E.B[0] + y * E.B[1] + z * E.B[2]);
    if (Hd) de += -0.5 * mu0 * E.V * Ms * (x * Hd[3 * nat] + y * Hd[3 * nat + 1] + z * Hd[3 * nat + 2]);
  }
  double vals[6] = {ex, dm, an, ze, lo, de};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k2 = 0; k2 < 6; ++k2) {
    const double w = warp_sum(vals[k2]);
    if (lane == 0) red[warp][k2] = w;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double acc = 0;
    for (int w = 0; w < kReduceBlock / 32; ++w) acc += red[w][threadIdx.x];
    part[8LL * blockIdx.x + threadIdx.x] = acc;
  }
}

__global__ void k_energy_final(const double *part, int nblocks, double *out7) {
  __shared__ double red[6][32];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 6; ++k) acc[k] += part[8LL * b + k];
  for (int k = 0; k < 6; ++k) {
    const double w = warp_sum(acc[k]);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0;
    for (int k = 0; k < 6; ++k) {
      double s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[k][w];
      out7[k + 1] = s;
      tot += s;
    }
    out7[0] = tot;
  }
}

void launch_energy(const Launch &L, const ChainDev *chains_d, int c, long long ncells_slots,
                   const float4 *m, const double *etab, const double *Hd, const EnergyCoef &E,
                   double *part, double *out7) {
  const int nb = (int)((2 * ncells_slots + kReduceBlock * 4 - 1) / (kReduceBlock * 4));
  k_energy_partial<<<nb, kReduceBlock, 0, L.stream>>>(chains_d, c, m, etab, Hd, E, part);
  k_energy_final<<<1, 256, 0, L.stream>>>(part, nb, out7);
  *L.counter += 2;
}

// ---------------------------------------------------------------------------
// natural <-> split copies of one chain; w (grain id) of the split array is kept
__global__ void k_pack(const ChainDev *chains, int c, float4 *m, const float4 *nat, int to_split) {
  const ChainDev &ch = chains[c];
  const long long S2 = 2LL * ch.nrows * ch.hx;
  const long long q2 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q2 >= S2) return;
  int color, i, row;
  long long q;
  if (!slot_cell(ch, q2, color, q, i, row)) return;
  const long long n = i + (long long)ch.nx * row;
  float4 *dst = m + ch.m_off + q2;
  if (to_split) {
    const float4 v = nat[n];
    *dst = make_float4(v.x, v.y, v.z, dst->w);
  } else {
    const float4 v = *dst;
    const_cast<float4 *>(nat)[n] = make_float4(v.x, v.y, v.z, 0.f);
  }
}

// flag = 1 if any of the first three components of v[0..n) is not finite
__global__ void k_check_finite(const float4 *v, long long n, int *flag) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const float4 a = v[q];
    if (!isfinite(a.x) || !isfinite(a.y) || !isfinite(a.z)) *flag = 1;
  }
}

void launch_check_finite(const Launch &L, const float4 *v, long long n, int *flag) {
  long long nb = (n + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  k_check_finite<<<(int)(nb < 1 ? 1 : nb), 256, 0, L.stream>>>(v, n, flag);
  ++*L.counter;
}

void launch_pack(const Launch &L, const ChainDev *chains_d, int c, long long slots, float4 *m,
                 const float4 *nat, int to_split) {
  const int nb = (int)((2 * slots + 255) / 256);
  k_pack<<<nb, 256, 0, L.stream>>>(chains_d, c, m, nat, to_split);
  ++*L.counter;
}

// random directions from Philox counter (cell, 0, chain, 1)
__global__ void k_init_random(const ChainDev *chains, int c, float4 *m, unsigned key0,
                              unsigned key1, const float *len_nat, float len) {
  const ChainDev &ch = chains[c];
  const long long S2 = 2LL * ch.nrows * ch.hx;
  const long long q2 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q2 >= S2) return;
  int color, i, row;
  long long q;
  if (!slot_cell(ch, q2, color, q, i, row)) return;
  const unsigned cell = (unsigned)(i + (long long)ch.nx * row);
  const uint4 r = philox4x32_10(make_uint4(cell, 0u, (unsigned)ch.chain, 1u), make_uint2(key0, key1));
  const float z = 2.f * uniform01(r.x) - 1.f;
  float sp, cp;
  sincospif(2.f * uniform01(r.y), &sp, &cp);
  const float rr = sqrtf(fmaxf(0.f, 1.f - z * z));
  const float L = len_nat ? len_nat[cell] : len;
  float4 *dst = m + ch.m_off + q2;
  *dst = make_float4(L * rr * cp, L * rr * sp, L * z, dst->w);
}

void launch_init_random(const Launch &L, const ChainDev *chains_d, int c, long long slots, float4 *m,
                        unsigned key0, unsigned key1, const float *len_nat, float len) {
  const int nb = (int)((2 * slots + 255) / 256);
  k_init_random<<<nb, 256, 0, L.stream>>>(chains_d, c, m, key0, key1, len_nat, len);
  ++*L.counter;
}

}  // namespace mmc
