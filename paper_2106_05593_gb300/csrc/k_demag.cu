// Demagnetizing field by FFT convolution with the Newell tensor (Sec. III,
// Eq. 14): H_d = -IFFT( N^ . FFT(Ms0 m) ), for every chain of a batch.  Open
// axes are zero padded to Px >= 2 nx; periodic demag axes either use the
// periodic kernel on the padded grid or, for power-of-two extents, a circular
// transform of length nx (ChainDev::circ).  This file holds the generic kernels
// (any nz, used for 3D meshes) and the dispatch; the interleaved 2D kernels are
// in k_demag_il.cuh.
//
// Three kernels per update, each batched over chains:
//  rows_fwd  two rows per sequence pair: the real rows Mx, My of row r, of row
//            r+1, and (Mz_r, Mz_{r+1}) are packed as three complex sequences,
//            zero padded to Px, transformed, and split into the half spectra
//            (kx in [0, Px/2]) of the six real rows.  Output: spectrum buffer
//            S[comp][row][kx] (row-major, stride Sx).
//  cols      C adjacent kx columns per block: FFT along y (and z), pointwise
//            H^ = -N^ M^ with the real tensor spectra (symmetric quadrant),
//            inverse transforms, rows outside the mesh dropped; in place in S.
//  rows_inv  inverse row transforms (two real rows per complex sequence),
//            crop to nx, scale by 1/(Px Py Pz), and write the sweep's static
//            field h_eff = zee (B + mu0 H_d) in the split layout, optionally
//            also H_d in FP64, natural order.
// The FFTs are the shared-memory Stockham transforms of fft.cuh; R = float,
// double or ff (float-float, ff.cuh) selects the arithmetic of the whole
// convolution.  The float-float convolution always takes these kernels, also
// for 2D chains.
#include <type_traits>

#include "demag_args.cuh"
#include "demag_il.h"
#include "ff.cuh"
#include "fft_il.cuh"

namespace mmc {

// the plans launch the generic kernels with at most this many threads
constexpr int kGenericThreads = 512;

template <typename R>
__global__ void __launch_bounds__(kGenericThreads) k_rows_fwd(DemagArgs<R> A) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  const int c = demag_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int Px = ch.Px, lx = ch.lx, nx = ch.nx, nrows = ch.nrows, Sx = ch.Sx;
  const int np = pairs_per_block(Px);
  const int pair0 = (int)(blockIdx.x - A.blk_first[c]) * np;
  const int totpairs = (nrows + 1) / 2;
  for (int idx = threadIdx.x; idx < np * Px; idx += blockDim.x) {
    const int qq = idx >> lx, x = idx & (Px - 1);
    const int pr = pair0 + qq, r0 = 2 * pr, r1 = r0 + 1;
    R M0x = 0, M0y = 0, M0z = 0, M1x = 0, M1y = 0, M1z = 0;
    if (pr < totpairs && x < nx) {
      if (A.m_nat) {
        const R Ms = A.Ms_override;
        const R *v0 = A.m_nat + 3 * ((long long)r0 * nx + x);
        M0x = Ms * v0[0]; M0y = Ms * v0[1]; M0z = Ms * v0[2];
        if (r1 < nrows) {
          const R *v1 = A.m_nat + 3 * ((long long)r1 * nx + x);
          M1x = Ms * v1[0]; M1y = Ms * v1[1]; M1z = Ms * v1[2];
        }
      } else {
        load_M<R>(ch, A.m, A.ms, A.ms_lo, r0, x, M0x, M0y, M0z, A.ck);
        if (r1 < nrows) load_M<R>(ch, A.m, A.ms, A.ms_lo, r1, x, M1x, M1y, M1z, A.ck);
      }
    }
    C z;
    z.x = M0x; z.y = M0y; buf[(3 * qq + 0) * Px + x] = z;
    z.x = M1x; z.y = M1y; buf[(3 * qq + 1) * Px + x] = z;
    z.x = M0z; z.y = M1z; buf[(3 * qq + 2) * Px + x] = z;
  }
  __syncthreads();
  fft_smem<C>(buf, lx, 3 * np, SeqMap{1, Px, 0, 1}, A.tw, false);
  const int half = Px / 2 + 1;
  const long long plane = (long long)nrows * Sx;
  C *S = A.S + ch.s_off;
  for (int idx = threadIdx.x; idx < np * half; idx += blockDim.x) {
    const int qq = idx / half, kx = idx - qq * half;
    const int pr = pair0 + qq, r0 = 2 * pr, r1 = r0 + 1;
    if (pr >= totpairs) continue;
    const int km = (Px - kx) & (Px - 1);
#pragma unroll
    for (int sq = 0; sq < 3; ++sq) {
      const C Z = buf[(3 * qq + sq) * Px + kx], Zm = buf[(3 * qq + sq) * Px + km];
      // a = (Z + conj(Zm)) / 2, b = (Z - conj(Zm)) / (2i)
      C a, b;
      a.x = (R)0.5 * (Z.x + Zm.x); a.y = (R)0.5 * (Z.y - Zm.y);
      b.x = (R)0.5 * (Z.y + Zm.y); b.y = (R)0.5 * (Zm.x - Z.x);
      if (sq == 0) {
        S[MMC_CK(A.ck, 0 * plane + (long long)r0 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)] = a;
        S[MMC_CK(A.ck, 1 * plane + (long long)r0 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)] = b;
      } else if (sq == 1) {
        if (r1 < nrows) {
          S[MMC_CK(A.ck, 0 * plane + (long long)r1 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)] = a;
          S[MMC_CK(A.ck, 1 * plane + (long long)r1 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)] = b;
        }
      } else {
        S[MMC_CK(A.ck, 2 * plane + (long long)r0 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)] = a;
        if (r1 < nrows) S[MMC_CK(A.ck, 2 * plane + (long long)r1 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)] = b;
      }
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kGenericThreads) k_cols(DemagArgs<R> A, int CC) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  const int c = demag_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int Px = ch.Px, Py = ch.Py, Pz = ch.Pz, ly = ch.ly, lz = ch.lz;
  const int ny = ch.ny, nz = ch.nz, nrows = ch.nrows, Sx = ch.Sx;
  const int kx0 = (int)(blockIdx.x - A.blk_first[c]) * CC;
  const int ncolq = Px / 2 + 1;
  const int PyPz = Py * Pz;
  const long long plane = (long long)nrows * Sx;
  C *S = A.S + ch.s_off;
  const int tot = 3 * CC * PyPz;
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) { buf[idx].x = 0; buf[idx].y = 0; }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 3 * nrows * CC; idx += blockDim.x) {
    const int col = idx % CC, rest = idx / CC;
    const int r = rest % nrows, comp = rest / nrows;
    const int kx = kx0 + col;
    if (kx < ncolq) {
      const int j = r % ny, k = r / ny;
      buf[((comp * CC + col) * Pz + k) * Py + j] = S[MMC_CK(A.ck, comp * plane + (long long)r * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)];
    }
  }
  __syncthreads();
  fft_smem<C>(buf, ly, 3 * CC * nz, SeqMap{nz, PyPz, Py, 1}, A.tw, false);
  if (Pz > 1) fft_smem<C>(buf, lz, 3 * CC * Py, SeqMap{Py, PyPz, 1, Py}, A.tw, false);
  // pointwise H^ = -N^ M^ with the real quadrant spectra
  const int qx = Px / 2 + 1, qy = Py / 2 + 1, qz = Pz / 2 + 1;
  const long long Q = (long long)qx * qy * qz;
  const R *nh = A.nhat[ch.spec];
  for (int idx = threadIdx.x; idx < CC * PyPz; idx += blockDim.x) {
    const int col = idx / PyPz, rem = idx - col * PyPz;
    const int kz = rem / Py, ky = rem - kz * Py;
    const int kx = kx0 + col;
    if (kx >= ncolq) continue;
    const int kyq = ky <= Py / 2 ? ky : Py - ky;
    const int kzq = kz <= Pz / 2 ? kz : Pz - kz;
    const R sy = ky <= Py / 2 ? (R)1 : (R)-1;
    const R sz = kz <= Pz / 2 ? (R)1 : (R)-1;
    const long long qi = MMC_CK(A.ck, ((long long)kzq * qy + kyq) * qx + kx, 0, Q, kCkDemagTensor);
    const R Nxx = nh[qi], Nyy = nh[Q + qi], Nzz = nh[2 * Q + qi], Nxy = sy * nh[3 * Q + qi];
    R Nxz = 0, Nyz = 0;
    if (Pz > 1) { Nxz = sz * nh[4 * Q + qi]; Nyz = sy * sz * nh[5 * Q + qi]; }
    const int b0 = ((0 * CC + col) * Pz + kz) * Py + ky;
    const int b1 = ((1 * CC + col) * Pz + kz) * Py + ky;
    const int b2 = ((2 * CC + col) * Pz + kz) * Py + ky;
    const C Mx = buf[b0], My = buf[b1], Mz = buf[b2];
    C hx_, hy_, hz_;
    hx_.x = -(Nxx * Mx.x + Nxy * My.x + Nxz * Mz.x);
    hx_.y = -(Nxx * Mx.y + Nxy * My.y + Nxz * Mz.y);
    hy_.x = -(Nxy * Mx.x + Nyy * My.x + Nyz * Mz.x);
    hy_.y = -(Nxy * Mx.y + Nyy * My.y + Nyz * Mz.y);
    hz_.x = -(Nxz * Mx.x + Nyz * My.x + Nzz * Mz.x);
    hz_.y = -(Nxz * Mx.y + Nyz * My.y + Nzz * Mz.y);
    buf[b0] = hx_; buf[b1] = hy_; buf[b2] = hz_;
  }
  __syncthreads();
  if (Pz > 1) fft_smem<C>(buf, lz, 3 * CC * Py, SeqMap{Py, PyPz, 1, Py}, A.tw, true);
  fft_smem<C>(buf, ly, 3 * CC * nz, SeqMap{nz, PyPz, Py, 1}, A.tw, true);
  for (int idx = threadIdx.x; idx < 3 * nrows * CC; idx += blockDim.x) {
    const int col = idx % CC, rest = idx / CC;
    const int r = rest % nrows, comp = rest / nrows;
    const int kx = kx0 + col;
    if (kx < ncolq) {
      const int j = r % ny, k = r / ny;
      S[MMC_CK(A.ck, comp * plane + (long long)r * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)] = buf[((comp * CC + col) * Pz + k) * Py + j];
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kGenericThreads) k_rows_inv(DemagArgs<R> A) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *buf = reinterpret_cast<C *>(smem_raw);
  const int c = demag_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int Px = ch.Px, lx = ch.lx, nx = ch.nx, nrows = ch.nrows, Sx = ch.Sx;
  const int np = pairs_per_block(Px);
  const int pair0 = (int)(blockIdx.x - A.blk_first[c]) * np;
  const int totpairs = (nrows + 1) / 2;
  const int half = Px / 2 + 1;
  const long long plane = (long long)nrows * Sx;
  const C *S = A.S + ch.s_off;
  for (int idx = threadIdx.x; idx < np * half; idx += blockDim.x) {
    const int qq = idx / half, kx = idx - qq * half;
    const int pr = pair0 + qq, r0 = 2 * pr, r1 = r0 + 1;
    C a[3], b[3];
    for (int t = 0; t < 3; ++t) { a[t].x = 0; a[t].y = 0; b[t] = a[t]; }
    if (pr < totpairs) {
      a[0] = S[MMC_CK(A.ck, 0 * plane + (long long)r0 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)];
      b[0] = S[MMC_CK(A.ck, 1 * plane + (long long)r0 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)];
      a[2] = S[MMC_CK(A.ck, 2 * plane + (long long)r0 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)];
      if (r1 < nrows) {
        a[1] = S[MMC_CK(A.ck, 0 * plane + (long long)r1 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)];
        b[1] = S[MMC_CK(A.ck, 1 * plane + (long long)r1 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)];
        b[2] = S[MMC_CK(A.ck, 2 * plane + (long long)r1 * Sx + kx, 0, spectrum_elems(ch), kCkDemagSpectrum)];
      }
    }
    const bool edge = (kx == 0) || (2 * kx == Px);
#pragma unroll
    for (int sq = 0; sq < 3; ++sq) {
      // z = a + i b for two real rows with Hermitian half spectra a, b
      C zk, zm;
      if (edge) {
        zk.x = a[sq].x; zk.y = b[sq].x;
        buf[(3 * qq + sq) * Px + kx] = zk;
      } else {
        zk.x = a[sq].x - b[sq].y; zk.y = a[sq].y + b[sq].x;
        zm.x = a[sq].x + b[sq].y; zm.y = b[sq].x - a[sq].y;
        buf[(3 * qq + sq) * Px + kx] = zk;
        buf[(3 * qq + sq) * Px + (Px - kx)] = zm;
      }
    }
  }
  __syncthreads();
  fft_smem<C>(buf, lx, 3 * np, SeqMap{1, Px, 0, 1}, A.tw, true);
  const R scale = (R)1 / ((R)Px * (R)ch.Py * (R)ch.Pz);
  const long long Sl = (long long)nrows * ch.hx;
  const bool percell = ch.t_off >= 0;
  const double mu0d = mu0;
  for (int idx = threadIdx.x; idx < np * nx; idx += blockDim.x) {
    const int qq = (int)divq((unsigned)idx, ch.nx_m, ch.nx_l), x = idx - qq * nx;
    const int pr = pair0 + qq;
    if (pr >= totpairs) continue;
    const C z0 = buf[(3 * qq + 0) * Px + x], z1 = buf[(3 * qq + 1) * Px + x], z2 = buf[(3 * qq + 2) * Px + x];
    for (int h = 0; h < 2; ++h) {
      const int r = 2 * pr + h;
      if (r >= nrows) break;
      const R Hx = (h == 0 ? z0.x : z1.x) * scale;
      const R Hy = (h == 0 ? z0.y : z1.y) * scale;
      const R Hz = (h == 0 ? z2.x : z2.y) * scale;
      const int j = r % ch.ny, k = r / ch.ny;
      const int colr = (x + j + k) & 1;
      const long long li = MMC_CK(A.ck, (long long)colr * Sl + (long long)r * ch.hx + (x >> 1), 0, 2 * Sl, kCkDemagField);
      if (A.heff) {
        const float zee = percell ? A.tab[ch.t_off + 2 * Sl + li].x : ch.zee;
        const float mu0f = (float)mu0d;
        A.heff[ch.h_off + li] = make_float4(zee * (ch.Bx + mu0f * (float)Hx), zee * (ch.By + mu0f * (float)Hy),
                                            zee * (ch.Bz + mu0f * (float)Hz), 0.f);
      }
      if (A.Hd && c == A.Hd_chain) {
        const long long nat = MMC_CK(A.ck, x + (long long)nx * r, 0, (long long)nx * nrows, kCkDemagField);
        A.Hd[3 * nat + 0] = (double)Hx;
        A.Hd[3 * nat + 1] = (double)Hy;
        A.Hd[3 * nat + 2] = (double)Hz;
      }
    }
  }
}

template <typename R>
void launch_demag_impl(const Launch &L, const DemagLaunch &P) {
  using C = typename Cx<R>::T;
  DemagArgs<R> A;
  A.chains = P.chains; A.m = P.m; A.tab = P.tab; A.ms = P.ms; A.ms_lo = P.ms_lo;
  A.S = reinterpret_cast<C *>(P.spec);
  A.nhat = reinterpret_cast<const R *const *>(P.nhat);
  A.tw = reinterpret_cast<const C *>(P.twiddle);
  A.heff = P.heff; A.Hd = P.Hd; A.Hd_chain = P.Hd_chain;
  A.m_nat = reinterpret_cast<const R *>(P.m_nat);
  A.Ms_override = (R)P.Ms_override;
  A.ck = P.ck;
  A.nchains = P.nchains;
  if constexpr (!std::is_same<R, ff>::value) {
    if (P.il2d) {
      if constexpr (sizeof(R) == 8) launch_il<CfgD16>(L, P, A);
      else if (P.fft_variant == 2) launch_il<CfgF32>(L, P, A);
      else if (P.fft_variant == 3) launch_il<CfgF16h>(L, P, A);
      else launch_il<CfgF16>(L, P, A);
      return;
    }
  }
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  if (P.ev) cudaEventRecord(P.ev[0], L.stream);
  k_rows_fwd<R><<<P.rows_blocks, P.rows_threads, P.rows_smem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[1], L.stream);
  A.blk_chain = P.cols_chain; A.blk_first = P.cols_first;
  k_cols<R><<<P.cols_blocks, P.cols_threads, P.cols_smem, L.stream>>>(A, P.cols_per_block);
  if (P.ev) cudaEventRecord(P.ev[2], L.stream);
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  k_rows_inv<R><<<P.rows_blocks, P.rows_threads, P.rows_smem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[3], L.stream);
  *L.counter += 3;
}

void launch_demag(const Launch &L, const DemagLaunch &P, bool fp64) {
  if (fp64 && P.ff) launch_demag_impl<ff>(L, P);
  else if (fp64) launch_demag_impl<double>(L, P);
  else if (P.w32) launch_w32(L, P);
  else launch_demag_impl<float>(L, P);
}

cudaError_t demag_set_smem_limits() {
  cudaError_t e = cudaSuccess;
  const int lim = 200 * 1024;
  e = cudaFuncSetAttribute(k_rows_fwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rows_fwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cols<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cols<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rows_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rows_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rows_fwd<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cols<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rows_inv<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e != cudaSuccess) return e;
  const int lil = 200 * 1024;
  if ((e = il_set_smem<CfgF16>(lil)) != cudaSuccess) return e;
  if ((e = il_set_smem<CfgF32>(lil)) != cudaSuccess) return e;
  if ((e = il_set_smem<CfgD16>(lil)) != cudaSuccess) return e;
  if ((e = w32_set_smem()) != cudaSuccess) return e;
  return il_set_smem<CfgF16h>(lil);
}

int il_elements(bool fp64) { return fp64 ? CfgD16::E : CfgF16::E; }
int il_padded_elements(bool fp64) { return il_padded(il_elements(fp64)); }
int il_elements_small() { return CfgF16h::E; }
int il_padded_of(int e) { return il_padded(e); }

}  // namespace mmc
