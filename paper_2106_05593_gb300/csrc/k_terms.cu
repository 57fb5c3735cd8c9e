// Size of each free-energy term of the trial moves (App. B, Fig. 11): for every
// cell of one chain (both sublattices, each against the same state and the
// frozen field h_eff of that state) the trial move the sweep would draw at
// iteration `sweep` is formed with the sweep's own pieces (trial.cuh), its
// energy change split into exchange, DMI, anisotropy, Zeeman, longitudinal and
// demag (Eq. 14) parts, and |part| (units of the cell's kT) summed in FP64.  The
// state is not changed.  Per-block partials are added in a fixed order, so the
// result does not depend on the schedule.
#include "philox.cuh"
#include "terms.h"
#include "trial.cuh"

namespace mmc {

constexpr int kTermsBlock = 256;

template <bool PERCELL>
__global__ void __launch_bounds__(kTermsBlock) k_trial_terms(const ChainDev *chains, const ChainState *st, int c,
                                                             const float4 *m, const float4 *heff, const float4 *tab,
                                                             unsigned sweep, unsigned key0, unsigned key1,
                                                             float omc_override, double *part) {
  const ChainK K = load_chain(chains + c);
  const int nx = K.nx, ny = K.ny, nz = K.nz, hx = K.hx;
  const unsigned S32 = (unsigned)K.nrows * (unsigned)hx;
  const long long S = (long long)S32;
  const float omc = omc_override >= 0.f ? omc_override : st[c].omc;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * S32; t += gridDim.x * blockDim.x) {
    const int color = t >= S32 ? 1 : 0;
    const unsigned q32 = t - (color ? S32 : 0u);
    const int row = (int)divq(q32, K.hx_m, K.hx_l);
    const int s = (int)(q32 - (unsigned)row * (unsigned)hx);
    const int k = (int)divq((unsigned)row, K.ny_m, K.ny_l), j = row - k * ny;
    const int p = (j + k + color) & 1;
    const int i = 2 * s + p;
    if (i >= nx) continue;
    const float4 *mc = m + K.m_off + (long long)color * S;
    const float4 *mo = m + K.m_off + (long long)(1 - color) * S;
    const float4 a = mc[q32];
    float4 nb[6];
    float w[6];
    load_neighbours(K.pbc, (K.flags & F_GRAIN) != 0, K.gscale, nx, ny, nz, hx, mo, a, i, j, k, row, s, p, nb, w);
    const CellMat M = cell_material<PERCELL>(K, tab, S, (long long)color * S + q32);
    const float zx = M.zee * K.Bx, zy = M.zee * K.By, zz = M.zee * K.Bz;   // Zeeman part of h_eff
    float4 h = make_float4(zx, zy, zz, 0.f);
    if (K.flags & F_DEMAG) h = heff[K.h_off + (long long)color * S + q32];
    const unsigned cell = (unsigned)i + (unsigned)nx * (unsigned)row;
    const uint4 r = philox4x32_10(make_uint4(cell, sweep, (unsigned)K.chain, 0u), make_uint2(key0, key1));
    Move v = move_length(a, M.me2h, M.me2l);
    move_direction(v, a, M.sigma, omc, uniform01(r.x), uniform01(r.y), uniform01(r.z));
    const float fex = exchange_change(v, a, nb, w, K.wx * M.bs, K.wy * M.bs, K.wz * M.bs, nz > 1);
    const float fdmi = linear_change(v, nb, w, K.cdx * M.bs, K.cdy * M.bs, (K.flags & F_DMI) != 0, 0.f, 0.f, 0.f);
    const float fan = anisotropy_change(v, K.flags, M.k1, M.k2, M.ex, M.ey, M.ez);
    const float fzee = -(v.dmx * zx + v.dmy * zy + v.dmz * zz);
    const float flong = longitudinal_change(v, M.p2, M.p4);
    const float fdem = -(v.dmx * (h.x - zx) + v.dmy * (h.y - zy) + v.dmz * (h.z - zz));
    acc[0] += fabsf(fex);
    acc[1] += fabsf(fdmi);
    acc[2] += fabsf(fan);
    acc[3] += fabsf(fzee);
    acc[4] += fabsf(flong);
    acc[5] += fabsf(fdem);
  }
  __shared__ double red[6][kTermsBlock / 32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double x = acc[q];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[q][wp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double x = 0;
    for (int k = 0; k < kTermsBlock / 32; ++k) x += red[threadIdx.x][k];
    part[6 * blockIdx.x + threadIdx.x] = x;
  }
}

__global__ void k_trial_terms_final(const double *part, int nblocks, double *out) {
  if (blockIdx.x != 0 || threadIdx.x >= 6) return;
  double x = 0;
  for (int b = 0; b < nblocks; ++b) x += part[6 * b + threadIdx.x];
  out[threadIdx.x] = x;
}

int trial_terms_blocks(long long slots) {
  long long nb = (2 * slots + kTermsBlock - 1) / kTermsBlock;
  if (nb > 152 * 8) nb = 152 * 8;
  return (int)(nb < 1 ? 1 : nb);
}

void launch_trial_terms(const Launch &L, const ChainDev *chains, const ChainState *st, int c, long long slots,
                        bool percell, const float4 *m, const float4 *heff, const float4 *tab, unsigned sweep,
                        unsigned key0, unsigned key1, float omc_override, double *part, double *out) {
  const int nb = trial_terms_blocks(slots);
  if (percell)
    k_trial_terms<true><<<nb, kTermsBlock, 0, L.stream>>>(chains, st, c, m, heff, tab, sweep, key0, key1,
                                                           omc_override, part);
  else
    k_trial_terms<false><<<nb, kTermsBlock, 0, L.stream>>>(chains, st, c, m, heff, tab, sweep, key0, key1,
                                                            omc_override, part);
  k_trial_terms_final<<<1, 32, 0, L.stream>>>(part, nb, out);
  *L.counter += 2;
}

}  // namespace mmc
