// Demag convolution (Sec. III, Eq. 14) through cuFFT, the library comparison
// for the library's own shared-memory transforms: zero-padded real arrays of
// Ms0 m, batched R2C (D2Z) transforms per padded size, the same pointwise
// product with the real tensor spectra, C2R (Z2D), crop to the mesh and
// h_eff = zee (B + mu0 H_d).  Selected with mmc_options.demag_cufft.
#include <cufft.h>

#include "mmc_internal.h"

namespace mmc {

struct CfArgs {
  const ChainDev *chains;
  const int *chain_of;        // chain index per group slot
  int nchain;                 // chains in this size group
  int Px, Py, Pz;
  const float4 *m;
  const float *ms;
  const float4 *tab;
  float4 *heff;
  double *Hd;
  int Hd_slot;
};

// padded real arrays [slot][comp][z][y][x]
template <typename R>
__global__ void k_cf_pad(CfArgs A, R *real) {
  const long long P = (long long)A.Px * A.Py * A.Pz;
  const long long tot = (long long)A.nchain * P;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int slot = (int)(t / P);
    const long long e = t - (long long)slot * P;
    const int x = (int)(e % A.Px);
    const int y = (int)((e / A.Px) % A.Py);
    const int z = (int)(e / ((long long)A.Px * A.Py));
    const ChainDev &ch = A.chains[A.chain_of[slot]];
    R mx = 0, my = 0, mz = 0;
    if (x < ch.nx && y < ch.ny && z < ch.nz) {
      const int r = y + ch.ny * z;
      const int col = (x + y + z) & 1;
      const long long S = (long long)ch.nrows * ch.hx;
      const long long idx = (long long)col * S + (long long)r * ch.hx + (x >> 1);
      const float4 v = A.m[ch.m_off + idx];
      const R Ms = ch.ms_off >= 0 ? (R)A.ms[ch.ms_off + idx] : (R)ch.Ms0d;
      mx = Ms * (R)v.x; my = Ms * (R)v.y; mz = Ms * (R)v.z;
    }
    R *b = real + (long long)slot * 3 * P + e;
    b[0] = mx;
    b[P] = my;
    b[2 * P] = mz;
  }
}

// H^ = -N^ M^ on the half spectra [slot][comp][kz][ky][kx], kx in [0, Px/2]
template <typename R, typename C>
__global__ void k_cf_mul(CfArgs A, C *cplx, const R *const *nhat) {
  const int qx = A.Px / 2 + 1, qy = A.Py / 2 + 1, qz = A.Pz / 2 + 1;
  const long long H = (long long)qx * A.Py * A.Pz;
  const long long Q = (long long)qx * qy * qz;
  const long long tot = (long long)A.nchain * H;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int slot = (int)(t / H);
    const long long e = t - (long long)slot * H;
    const int kx = (int)(e % qx);
    const int ky = (int)((e / qx) % A.Py);
    const int kz = (int)(e / ((long long)qx * A.Py));
    const ChainDev &ch = A.chains[A.chain_of[slot]];
    const R *nh = nhat[ch.spec];
    const int kyq = ky <= A.Py / 2 ? ky : A.Py - ky;
    const int kzq = kz <= A.Pz / 2 ? kz : A.Pz - kz;
    const R sy = ky <= A.Py / 2 ? (R)1 : (R)-1;
    const R sz = kz <= A.Pz / 2 ? (R)1 : (R)-1;
    const long long qi = ((long long)kzq * qy + kyq) * qx + kx;
    const R Nxx = nh[qi], Nyy = nh[Q + qi], Nzz = nh[2 * Q + qi], Nxy = sy * nh[3 * Q + qi];
    R Nxz = 0, Nyz = 0;
    if (A.Pz > 1) { Nxz = sz * nh[4 * Q + qi]; Nyz = sy * sz * nh[5 * Q + qi]; }
    C *b = cplx + (long long)slot * 3 * H + e;
    const C Mx = b[0], My = b[H], Mz = b[2 * H];
    C hx, hy, hz;
    hx.x = -(Nxx * Mx.x + Nxy * My.x + Nxz * Mz.x);
    hx.y = -(Nxx * Mx.y + Nxy * My.y + Nxz * Mz.y);
    hy.x = -(Nxy * Mx.x + Nyy * My.x + Nyz * Mz.x);
    hy.y = -(Nxy * Mx.y + Nyy * My.y + Nyz * Mz.y);
    hz.x = -(Nxz * Mx.x + Nyz * My.x + Nzz * Mz.x);
    hz.y = -(Nxz * Mx.y + Nyz * My.y + Nzz * Mz.y);
    b[0] = hx;
    b[H] = hy;
    b[2 * H] = hz;
  }
}

template <typename R>
__global__ void k_cf_crop(CfArgs A, const R *real) {
  const long long P = (long long)A.Px * A.Py * A.Pz;
  const long long tot = (long long)A.nchain * P;
  const R scale = (R)1 / (R)P;
  const float mu0f = (float)mu0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int slot = (int)(t / P);
    const long long e = t - (long long)slot * P;
    const int x = (int)(e % A.Px);
    const int y = (int)((e / A.Px) % A.Py);
    const int z = (int)(e / ((long long)A.Px * A.Py));
    const ChainDev &ch = A.chains[A.chain_of[slot]];
    if (x >= ch.nx || y >= ch.ny || z >= ch.nz) continue;
    const R *b = real + (long long)slot * 3 * P + e;
    const R Hx = b[0] * scale, Hy = b[P] * scale, Hz = b[2 * P] * scale;
    const int r = y + ch.ny * z;
    const int col = (x + y + z) & 1;
    const long long S = (long long)ch.nrows * ch.hx;
    const long long li = (long long)col * S + (long long)r * ch.hx + (x >> 1);
    if (A.heff) {
      const float zee = ch.t_off >= 0 ? A.tab[ch.t_off + 2 * S + li].x : ch.zee;
      A.heff[ch.h_off + li] = make_float4(zee * (ch.Bx + mu0f * (float)Hx), zee * (ch.By + mu0f * (float)Hy),
                                          zee * (ch.Bz + mu0f * (float)Hz), 0.f);
    }
    if (A.Hd && slot == A.Hd_slot) {
      const long long nat = x + (long long)ch.nx * r;
      A.Hd[3 * nat] = (double)Hx;
      A.Hd[3 * nat + 1] = (double)Hy;
      A.Hd[3 * nat + 2] = (double)Hz;
    }
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_cufft_group(const Launch &L, const CufftGroup &G, const ChainDev *chains_d,
                               const float4 *m, const float *ms, const float4 *tab, float4 *heff,
                               double *Hd, int Hd_slot, const void *const *nhat, cudaEvent_t *ev) {
  CfArgs A;
  A.chains = chains_d;
  A.chain_of = G.chain_of;
  A.nchain = G.nchain;
  A.Px = G.Px; A.Py = G.Py; A.Pz = G.Pz;
  A.m = m; A.ms = ms; A.tab = tab; A.heff = heff; A.Hd = Hd; A.Hd_slot = Hd_slot;
  const long long P = (long long)G.Px * G.Py * G.Pz;
  const long long H = (long long)(G.Px / 2 + 1) * G.Py * G.Pz;
  const int gp = grid_for((long long)G.nchain * P), gh = grid_for((long long)G.nchain * H);
  if (cufftSetStream(G.fwd, L.stream) != CUFFT_SUCCESS || cufftSetStream(G.inv, L.stream) != CUFFT_SUCCESS)
    return cudaErrorUnknown;
  if (ev) cudaEventRecord(ev[0], L.stream);
  cufftResult r;
  if (G.fp64) {
    k_cf_pad<double><<<gp, 256, 0, L.stream>>>(A, (double *)G.real);
    r = cufftExecD2Z(G.fwd, (cufftDoubleReal *)G.real, (cufftDoubleComplex *)G.cplx);
    if (ev) cudaEventRecord(ev[1], L.stream);
    k_cf_mul<double, double2><<<gh, 256, 0, L.stream>>>(A, (double2 *)G.cplx, (const double *const *)nhat);
    if (ev) cudaEventRecord(ev[2], L.stream);
    if (r == CUFFT_SUCCESS) r = cufftExecZ2D(G.inv, (cufftDoubleComplex *)G.cplx, (cufftDoubleReal *)G.real);
    k_cf_crop<double><<<gp, 256, 0, L.stream>>>(A, (const double *)G.real);
  } else {
    k_cf_pad<float><<<gp, 256, 0, L.stream>>>(A, (float *)G.real);
    r = cufftExecR2C(G.fwd, (cufftReal *)G.real, (cufftComplex *)G.cplx);
    if (ev) cudaEventRecord(ev[1], L.stream);
    k_cf_mul<float, float2><<<gh, 256, 0, L.stream>>>(A, (float2 *)G.cplx, (const float *const *)nhat);
    if (ev) cudaEventRecord(ev[2], L.stream);
    if (r == CUFFT_SUCCESS) r = cufftExecC2R(G.inv, (cufftComplex *)G.cplx, (cufftReal *)G.real);
    k_cf_crop<float><<<gp, 256, 0, L.stream>>>(A, (const float *)G.real);
  }
  if (ev) cudaEventRecord(ev[3], L.stream);
  *L.counter += 3;
  return r == CUFFT_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

cudaError_t make_cufft_plans(CufftGroup &G) {
  const int rank = G.Pz > 1 ? 3 : 2;
  int n3[3] = {G.Pz, G.Py, G.Px};
  int n2[2] = {G.Py, G.Px};
  int *n = rank == 3 ? n3 : n2;
  const int batch = 3 * G.nchain;
  const long long P = (long long)G.Px * G.Py * G.Pz;
  const long long H = (long long)(G.Px / 2 + 1) * G.Py * G.Pz;
  cufftResult r = cufftPlanMany(&G.fwd, rank, n, nullptr, 1, (int)P, nullptr, 1, (int)H,
                                G.fp64 ? CUFFT_D2Z : CUFFT_R2C, batch);
  if (r != CUFFT_SUCCESS) return cudaErrorMemoryAllocation;
  r = cufftPlanMany(&G.inv, rank, n, nullptr, 1, (int)H, nullptr, 1, (int)P, G.fp64 ? CUFFT_Z2D : CUFFT_C2R, batch);
  if (r != CUFFT_SUCCESS) return cudaErrorMemoryAllocation;
  G.planned = true;
  return cudaSuccess;
}

void destroy_cufft_plans(CufftGroup &G) {
  if (G.planned) {
    cufftDestroy(G.fwd);
    cufftDestroy(G.inv);
    G.planned = false;
  }
}

}  // namespace mmc
