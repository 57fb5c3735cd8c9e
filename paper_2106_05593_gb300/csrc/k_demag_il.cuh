// Interleaved 2D demag kernels (Sec. III, Eq. 14): forward row transforms,
// column transforms with the tensor product, inverse row transforms with the
// crop and the sweep's field.  Included only by the per-configuration
// translation units k_demag_il_*.cu, which instantiate launch_il and
// il_set_smem for one configuration each.
//
// A periodic demag axis whose extent is a power of two is transformed
// circularly (ChainDev::circ, length n, no zero padding, all outputs kept);
// every other axis is zero padded to Px >= 2 nx with the padding pruned (the
// first pass skips the zero upper half, the last pass stores only the crop).
#pragma once

#include "demag_il.h"
#include "fft_il.cuh"

namespace mmc {

// index of (comp, y, kx) in the column-tiled spectrum layout [comp][kx / CC][y][CC], CC = 2^lcc
__device__ __forceinline__ long long tiled(int comp, int y, int kx, int ny, int NG, int lcc) {
  return ((long long)(comp * NG + (kx >> lcc)) * ny + y) * (1 << lcc) + (kx & ((1 << lcc) - 1));
}

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

template <typename CFG>
__global__ void __launch_bounds__(CFG::E / CFG::V, CFG::MINB) k_rows_fwd2(DemagArgs<typename CFG::R> A) {
  using R = typename CFG::R;
  using C = typename Cx<R>::T;
  constexpr int E = CFG::E, V = CFG::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *raw = reinterpret_cast<C *>(smem_raw);
  C *buf = raw;
  const int c = demag_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int Px = ch.Px, lx = ch.lx, nx = ch.nx, ny = ch.ny, Sx = ch.Sx;
  // 3 groups (x+iy of the even row, x+iy of the odd row, z_even + i z_odd) of np
  // interleaved sequences: element (g, x, qq) at g * Px * np + x * np + qq
  constexpr int LE3 = ilog2c(E / 3);         // E / 3 is a power of two
  const int lnp = LE3 - lx, np = 1 << lnp, gs = Px * np;
  const int lcc = LE3 - ch.ly, CC = 1 << lcc, NG = Sx >> lcc;
  const int pair0 = (int)(blockIdx.x - A.blk_first[c]) * np;
  const int totpairs = (ny + 1) / 2;
  C *tws = raw + il_padded(E);               // pass twiddle tables (at most Px entries)
  il_twiddles<C, V>(tws, A.tw, lx);
  // Padded rows: the upper half x >= Px/2 is zero padding the first FFT pass
  // never reads.  Circular rows (x periodic, Px = nx): the whole row.
  const bool circ = (ch.circ & 1) != 0;
  const int lfill = circ ? lx : lx - 1;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < (np << lfill); idx += blockDim.x) {
    const int qq = idx >> lfill, x = idx & ((1 << lfill) - 1);
    const int pr = pair0 + qq, r0 = 2 * pr, r1 = r0 + 1;
    R M0x = 0, M0y = 0, M0z = 0, M1x = 0, M1y = 0, M1z = 0;
    if (pr < totpairs && x < nx) {
      if (A.m_nat) {
        const R Ms = A.Ms_override;
        const R *v0 = A.m_nat + 3 * ((long long)r0 * nx + x);
        M0x = Ms * v0[0]; M0y = Ms * v0[1]; M0z = Ms * v0[2];
        if (r1 < ny) {
          const R *v1 = A.m_nat + 3 * ((long long)r1 * nx + x);
          M1x = Ms * v1[0]; M1y = Ms * v1[1]; M1z = Ms * v1[2];
        }
      } else {
        load_M<R>(ch, A.m, A.ms, A.ms_lo, r0, x, M0x, M0y, M0z, A.ck);
        if (r1 < ny) load_M<R>(ch, A.m, A.ms, A.ms_lo, r1, x, M1x, M1y, M1z, A.ck);
      }
    }
    C z;
    const int e0 = x * np + qq;
    z.x = M0x; z.y = M0y; buf[e0] = z;
    z.x = M1x; z.y = M1y; buf[e0 + gs] = z;
    z.x = M0z; z.y = M1z; buf[e0 + 2 * gs] = z;
  }
  __syncthreads();
  if (circ) fft_il<C, V, false, false, false>(buf, lx, IlMap{lnp, 3, gs}, tws);
  else fft_il<C, V, false, true, false>(buf, lx, IlMap{lnp, 3, gs}, tws);
  // half spectra (kx <= Px/2) of the six real rows of each pair, written in
  // tiled order: c fastest, then the block's rows, then column group, then comp
  const int half = Px / 2 + 1;
  const int nrb = 2 * np, lnrb = lnp + 1;
  const int ngu = (half + CC - 1) / CC;
  C *S = A.S + ch.s_off;
  const int tot = 3 * ngu * nrb * CC;
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int cc = idx & (CC - 1), rr = (idx >> lcc) & (nrb - 1), o = idx >> (lcc + lnrb);
    const int comp = (o >= ngu) + (o >= 2 * ngu), g = o - comp * ngu;
    const int kx = g * CC + cc;
    const int r = 2 * pair0 + rr;
    if (kx >= half || r >= ny) continue;
    const int qq = rr >> 1, h = rr & 1;
    const int sq = comp == 2 ? 2 : h;
    const bool take_b = comp == 1 || (comp == 2 && h == 1);
    const int km = (Px - kx) & (Px - 1);
    const C Z = buf[sq * gs + kx * np + qq], Zm = buf[sq * gs + km * np + qq];
    C o2;
    if (!take_b) { o2.x = (R)0.5 * (Z.x + Zm.x); o2.y = (R)0.5 * (Z.y - Zm.y); }
    else { o2.x = (R)0.5 * (Z.y + Zm.y); o2.y = (R)0.5 * (Zm.x - Z.x); }
    S[MMC_CK(A.ck, tiled(comp, r, kx, ny, NG, lcc), 0, spectrum_elems(ch), kCkDemagSpectrum)] = o2;
  }
}

template <typename CFG>
__global__ void __launch_bounds__(CFG::E / CFG::V, CFG::MINB) k_cols2d(DemagArgs<typename CFG::R> A) {
  using R = typename CFG::R;
  using C = typename Cx<R>::T;
  constexpr int E = CFG::E, V = CFG::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *raw = reinterpret_cast<C *>(smem_raw);
  C *buf = raw;
  const int c = demag_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int Px = ch.Px, Py = ch.Py, ly = ch.ly, ny = ch.ny, Sx = ch.Sx;
  constexpr int LE3 = ilog2c(E / 3);         // E / 3 is a power of two
  const int lcc = LE3 - ly, CC = 1 << lcc, NG = Sx >> lcc;
  const int g = (int)(blockIdx.x - A.blk_first[c]);
  const int kx0 = g * CC;
  const int qx = Px / 2 + 1, qy = Py / 2 + 1;
  const C *S = A.S + ch.s_off;
  C *tws = raw + il_padded(E);               // pass twiddle tables (at most Py entries)
  il_twiddles<C, V>(tws, A.tw, ly);
  // buf[(comp * Py + y) * CC + cc]; padded columns: rows y >= ny are the zero
  // padding and the upper half y >= Py/2 is never read by the first FFT pass;
  // circular columns (y periodic, Py = ny): every row
  const bool circ = (ch.circ & 2) != 0;
  if (circ) {
#pragma unroll 8
    for (int idx = threadIdx.x; idx < E; idx += blockDim.x) {
      const int cc = idx & (CC - 1), y = (idx >> lcc) & (Py - 1), comp = idx >> LE3;
      buf[idx] = S[MMC_CK(A.ck, ((long long)(comp * NG + g) * ny + y) * CC + cc, 0, spectrum_elems(ch), kCkDemagSpectrum)];
    }
  } else {
#pragma unroll 8
    for (int idx = threadIdx.x; idx < E / 2; idx += blockDim.x) {
      const int cc = idx & (CC - 1), y = (idx >> lcc) & ((Py >> 1) - 1), comp = idx >> (LE3 - 1);
      C v;
      v.x = 0; v.y = 0;
      if (y < ny) v = S[MMC_CK(A.ck, ((long long)(comp * NG + g) * ny + y) * CC + cc, 0, spectrum_elems(ch), kCkDemagSpectrum)];
      buf[(comp * Py + y) * CC + cc] = v;
    }
  }
  __syncthreads();
  if (circ) fft_il<C, V, false, false, false>(buf, ly, IlMap{lcc, 3, Py * CC}, tws);
  else fft_il<C, V, false, true, false>(buf, ly, IlMap{lcc, 3, Py * CC}, tws);
  const long long Q = (long long)qx * qy;
  const R *nh = A.nhat[ch.spec];
  for (int idx = threadIdx.x; idx < Py * CC; idx += blockDim.x) {
    const int cc = idx & (CC - 1), ky = idx >> lcc;
    const int kx = kx0 + cc;
    if (kx >= qx) continue;
    const int kyq = ky <= Py / 2 ? ky : Py - ky;
    const R sy = ky <= Py / 2 ? (R)1 : (R)-1;
    const long long qi = MMC_CK(A.ck, (long long)kyq * qx + kx, 0, Q, kCkDemagTensor);
    const R Nxx = nh[qi], Nyy = nh[Q + qi], Nzz = nh[2 * Q + qi], Nxy = sy * nh[3 * Q + qi];
    const int b0 = ky * CC + cc, b1 = (Py + ky) * CC + cc, b2 = (2 * Py + ky) * CC + cc;
    const C Mx = buf[b0], My = buf[b1], Mz = buf[b2];
    C hx_, hy_, hz_;
    hx_.x = -(Nxx * Mx.x + Nxy * My.x);
    hx_.y = -(Nxx * Mx.y + Nxy * My.y);
    hy_.x = -(Nxy * Mx.x + Nyy * My.x);
    hy_.y = -(Nxy * Mx.y + Nyy * My.y);
    hz_.x = -(Nzz * Mz.x);
    hz_.y = -(Nzz * Mz.y);
    buf[b0] = hx_; buf[b1] = hy_; buf[b2] = hz_;
  }
  __syncthreads();
  if (circ) fft_il<C, V, true, false, false>(buf, ly, IlMap{lcc, 3, Py * CC}, tws);
  else fft_il<C, V, true, false, true>(buf, ly, IlMap{lcc, 3, Py * CC}, tws);
  C *So = A.S + ch.s_off;
  for (int idx = threadIdx.x; idx < E; idx += blockDim.x) {
    const int cc = idx & (CC - 1), y = (idx >> lcc) & (Py - 1), comp = idx >> LE3;
    if (y < ny) So[MMC_CK(A.ck, ((long long)(comp * NG + g) * ny + y) * CC + cc, 0, spectrum_elems(ch), kCkDemagSpectrum)] = buf[idx];
  }
}

template <typename CFG>
__global__ void __launch_bounds__(CFG::E / CFG::V, CFG::MINB) k_rows_inv2(DemagArgs<typename CFG::R> A) {
  using R = typename CFG::R;
  using C = typename Cx<R>::T;
  constexpr int E = CFG::E, V = CFG::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *raw = reinterpret_cast<C *>(smem_raw);
  C *buf = raw;
  const int c = demag_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int Px = ch.Px, lx = ch.lx, nx = ch.nx, ny = ch.ny, Sx = ch.Sx;
  constexpr int LE3 = ilog2c(E / 3);         // E / 3 is a power of two
  const int lnp = LE3 - lx, np = 1 << lnp, gs = Px * np;
  const int lcc = LE3 - ch.ly, CC = 1 << lcc, NG = Sx >> lcc;
  const int pair0 = (int)(blockIdx.x - A.blk_first[c]) * np;
  const int half = Px / 2 + 1;
  const int nrb = 2 * np, lnrb = lnp + 1;
  const int ngu = (half + CC - 1) / CC;
  const C *S = A.S + ch.s_off;
  C *tws = raw + il_padded(E);               // pass twiddle tables (at most Px entries)
  il_twiddles<C, V>(tws, A.tw, lx);
  // Each sequence is z = a + i b for the half spectra a, b of two real rows:
  // z[k] = a[k] + i b[k] and z[Px - k] = conj(a[k]) + i conj(b[k]), real parts only
  // at k = 0 and Px/2 (where the spectra of real rows are real).  Sequence
  // (h, qq) pairs x and y of row 2 qq + h, sequence (2, qq) the z of rows 2 qq and
  // 2 qq + 1; a work item (kx, row) reads its values and writes z directly.
  auto put = [&](int sb, int kx, C a, C b) {
    if (kx == 0 || 2 * kx == Px) {
      C z;
      z.x = a.x; z.y = b.x;
      buf[sb + kx * np] = z;
    } else {
      C zk, zm;
      zk.x = a.x - b.y; zk.y = a.y + b.x;
      zm.x = a.x + b.y; zm.y = b.x - a.y;
      buf[sb + kx * np] = zk;
      buf[sb + (Px - kx) * np] = zm;
    }
  };
  const int tot = ngu * nrb * CC;
#pragma unroll 8
  for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int cc = idx & (CC - 1), rr = (idx >> lcc) & (nrb - 1), g = idx >> (lcc + lnrb);
    const int kx = g * CC + cc;
    if (kx >= half) continue;
    const int r = 2 * pair0 + rr;
    const int qq = rr >> 1, h = rr & 1;
    C ax, ay, z0, z1;
    ax.x = ax.y = ay.x = ay.y = z0.x = z0.y = z1.x = z1.y = 0;
    if (r < ny) {
      const long long se = spectrum_elems(ch);
      ax = S[MMC_CK(A.ck, tiled(0, r, kx, ny, NG, lcc), 0, se, kCkDemagSpectrum)];
      ay = S[MMC_CK(A.ck, tiled(1, r, kx, ny, NG, lcc), 0, se, kCkDemagSpectrum)];
      if (h == 0) {
        z0 = S[MMC_CK(A.ck, tiled(2, r, kx, ny, NG, lcc), 0, se, kCkDemagSpectrum)];
        if (r + 1 < ny) z1 = S[MMC_CK(A.ck, tiled(2, r + 1, kx, ny, NG, lcc), 0, se, kCkDemagSpectrum)];
      }
    }
    put(h * gs + qq, kx, ax, ay);
    if (h == 0) put(2 * gs + qq, kx, z0, z1);
  }
  __syncthreads();
  // padded rows keep the lower half (the crop); circular rows keep every x
  if (ch.circ & 1) fft_il<C, V, true, false, false>(buf, lx, IlMap{lnp, 3, gs}, tws);
  else fft_il<C, V, true, false, true>(buf, lx, IlMap{lnp, 3, gs}, tws);
  const R scale = (R)1 / ((R)Px * (R)ch.Py * (R)ch.Pz);
  const long long Sl = (long long)ny * ch.hx;
  const bool percell = ch.t_off >= 0;
  const float mu0f = (float)mu0;
  const int totpairs = (ny + 1) / 2;
  for (int idx = threadIdx.x; idx < np * nx; idx += blockDim.x) {
    const int qq = (int)divq((unsigned)idx, ch.nx_m, ch.nx_l), x = idx - qq * nx;
    const int pr = pair0 + qq;
    if (pr >= totpairs) continue;
    const C z0 = buf[x * np + qq], z1 = buf[gs + x * np + qq], z2 = buf[2 * gs + x * np + qq];
    for (int h = 0; h < 2; ++h) {
      const int r = 2 * pr + h;
      if (r >= ny) break;
      const R Hx = (h == 0 ? z0.x : z1.x) * scale;
      const R Hy = (h == 0 ? z0.y : z1.y) * scale;
      const R Hz = (h == 0 ? z2.x : z2.y) * scale;
      const int colr = (x + r) & 1;
      const long long li = MMC_CK(A.ck, (long long)colr * Sl + (long long)r * ch.hx + (x >> 1), 0, 2 * Sl, kCkDemagField);
      if (A.heff) {
        const float zee = percell ? A.tab[ch.t_off + 2 * Sl + li].x : ch.zee;
        A.heff[ch.h_off + li] = make_float4(zee * (ch.Bx + mu0f * (float)Hx), zee * (ch.By + mu0f * (float)Hy),
                                            zee * (ch.Bz + mu0f * (float)Hz), 0.f);
      }
      if (A.Hd && c == A.Hd_chain) {
        const long long nat = MMC_CK(A.ck, x + (long long)nx * r, 0, (long long)nx * ny, kCkDemagField);
        A.Hd[3 * nat + 0] = (double)Hx;
        A.Hd[3 * nat + 1] = (double)Hy;
        A.Hd[3 * nat + 2] = (double)Hz;
      }
    }
  }
}

template <typename CFG>
void launch_il(const Launch &L, const DemagLaunch &P, DemagArgs<typename CFG::R> A) {
  using C = typename Cx<typename CFG::R>::T;
  constexpr int T = CFG::E / CFG::V;
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  if (P.ev) cudaEventRecord(P.ev[0], L.stream);
  k_rows_fwd2<CFG><<<P.rows_blocks, T, P.rows_smem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[1], L.stream);
  A.blk_chain = P.cols_chain; A.blk_first = P.cols_first;
  k_cols2d<CFG><<<P.cols_blocks, T, P.cols_smem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[2], L.stream);
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  k_rows_inv2<CFG><<<P.rows_blocks, T, P.inv_smem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[3], L.stream);
  *L.counter += 3;
}

template <typename CFG>
cudaError_t il_set_smem(int bytes) {
  const void *fns[3] = {(const void *)k_rows_fwd2<CFG>, (const void *)k_cols2d<CFG>,
                        (const void *)k_rows_inv2<CFG>};
  for (const void *f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace mmc
