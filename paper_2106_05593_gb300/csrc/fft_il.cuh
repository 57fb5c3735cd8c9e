// Interleaved shared-memory FFTs for the 2D demag convolution (Sec. III, Eq. 14).
//
// A block transforms `nseq` interleaved sequences in each of `ngroups` groups:
// element e of sequence (g, s) lives at buf[g * gstride + e * nseq + s], so
// threads that handle the same butterfly index of neighbouring sequences touch
// neighbouring shared-memory words and share one twiddle.  Each pass is a
// Stockham autosort radix-R step (R = 16 while possible, then 8, 4 or 2):
// every thread loads V complex values (V / R butterflies) into registers,
// all threads synchronize, then twiddle, transform and store them; a sequence of
// length N takes ceil(log16 N) passes.  The inverse pass is conj(F(conj(x))).
// Twiddles come from per-pass tables built from the FP64-built table
// tw[t] = exp(-2 pi i t / 4096), laid out so that the butterflies of one warp
// read neighbouring entries.
#pragma once

#include "fft.cuh"

namespace mmc {

// W16^m = exp(-2 pi i m / 16), m = 0..15
__device__ __forceinline__ void w16(int m, double &c, double &s) {
  const double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, H = 0.70710678118654752440;
  const double tc[16] = {1, C1, H, S1, 0, -S1, -H, -C1, -1, -C1, -H, -S1, 0, S1, H, C1};
  const double ts[16] = {0, -S1, -H, -C1, -1, -C1, -H, -S1, 0, S1, H, C1, 1, C1, H, S1};
  c = tc[m];
  s = ts[m];
}

template <typename C> __device__ __forceinline__ C cmul_w16(C a, int m) {
  using R = decltype(a.x);
  double cd, sd;
  w16(m, cd, sd);
  const R c = (R)cd, s = (R)sd;
  C r;
  r.x = a.x * c - a.y * s;
  r.y = a.x * s + a.y * c;
  return r;
}

// forward 16-point DFT in registers: 4 x 4 Cooley-Tukey (n = 4 n1 + n2, k = k1 + 4 k2)
template <typename C> __device__ __forceinline__ void dft16(C *x) {
  C a[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C t[4] = {x[n2], x[4 + n2], x[8 + n2], x[12 + n2]};
    dft4(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[4 * n2 + k1] = (n2 * k1) ? cmul_w16(t[k1], n2 * k1) : t[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C t[4] = {a[k1], a[4 + k1], a[8 + k1], a[12 + k1]};
    dft4(t);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = t[k2];
  }
}

// W32^m = exp(-2 pi i m / 32), m = 0..21 (the twiddles n2 k1 of a 4 x 8 split),
// cos and -sin of 2 pi m / 32 rounded to double; m is a compile-time constant
// after unrolling, so the selection folds away
template <typename C> __device__ __forceinline__ C cmul_w32(C a, int m) {
  using R = decltype(a.x);
  const double tc[22] = {1.0, 0.9807852804032304, 0.9238795325112867, 0.8314696123025452, 0.7071067811865476, 0.5555702330196023, 0.38268343236508984, 0.19509032201612833, 0.0, -0.1950903220161282, -0.3826834323650897, -0.555570233019602, -0.7071067811865475, -0.8314696123025453, -0.9238795325112867, -0.9807852804032304, -1.0, -0.9807852804032304, -0.9238795325112868, -0.8314696123025455, -0.7071067811865477, -0.5555702330196022};
  const double ts[22] = {0.0, -0.19509032201612825, -0.3826834323650898, -0.5555702330196022, -0.7071067811865475, -0.8314696123025452, -0.9238795325112867, -0.9807852804032304, -1.0, -0.9807852804032304, -0.9238795325112867, -0.8314696123025455, -0.7071067811865476, -0.5555702330196022, -0.3826834323650899, -0.1950903220161286, 0.0, 0.19509032201612836, 0.38268343236508967, 0.555570233019602, 0.7071067811865475, 0.8314696123025452};
  const R c = (R)tc[m], s = (R)ts[m];
  C r;
  r.x = a.x * c - a.y * s;
  r.y = a.x * s + a.y * c;
  return r;
}

// forward 32-point DFT in registers: 4 x 8 Cooley-Tukey (n = 8 n1 + n2, k = k1 + 4 k2)
template <typename C> __device__ __forceinline__ void dft32(C *x) {
  C a[32];
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2) {
    C t[4] = {x[n2], x[8 + n2], x[16 + n2], x[24 + n2]};
    dft4(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[4 * n2 + k1] = (n2 * k1) ? cmul_w32(t[k1], n2 * k1) : t[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C t[8] = {a[k1], a[4 + k1], a[8 + k1], a[12 + k1], a[16 + k1], a[20 + k1], a[24 + k1], a[28 + k1]};
    dft8(t);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) x[k1 + 4 * k2] = t[k2];
  }
}

template <typename C, int R> __device__ __forceinline__ void dft_r(C *u) {
  if (R == 32) dft32(u);
  else if (R == 16) dft16(u);
  else if (R == 8) dft8(u);
  else if (R == 4) dft4(u);
  else if (R == 2) dft2(u[0], u[1]);
}

// Bank padding: the stores of a first Stockham pass put neighbouring
// butterflies R * nseq elements apart, which maps many lanes of a warp to the
// same shared-memory bank.  That pass therefore writes, and the next pass reads,
// a layout with one padding element after every 2^kIlPad elements; all other
// passes, and the kernels around the transform, use the plain layout.
constexpr int kIlPad = 4;
template <bool PAD> __device__ __forceinline__ int il_at(int x) { return PAD ? x + (x >> kIlPad) : x; }
// elements a block buffer of e logical elements must hold (padded layout included)
__host__ __device__ constexpr int il_padded(int e) { return e + (e >> kIlPad) + 1; }

struct IlMap {
  int lnseq;        // log2 of the interleaved sequences per group (a power of two)
  int ngroups, gstride;
};

// one radix-R Stockham pass over all interleaved sequences (p = product of the
// radices already done); V values per thread.  ZIN (first pass only): the upper
// half of every sequence is known to be zero and is not read.  HALFOUT (last
// pass only): only the lower half of every output sequence is stored.  PIN /
// POUT: the input / output layout is the padded one.
template <typename C, int R, int V, bool INV, bool ZIN, bool HALFOUT, bool PIN, bool POUT, int TOFF>
__device__ __forceinline__ void il_pass(C *buf, int N, int p, IlMap mp, const C *__restrict__ tw) {
  constexpr int NB = V / R;
  const int nbf = N / R;              // compile-time: N and R are template constants
  const int nseq = 1 << mp.lnseq;
  const int total = mp.ngroups * (nbf << mp.lnseq);
  C v[V];
  int addr[NB], kk[NB];
  bool on[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int bf = threadIdx.x + i * blockDim.x;
    on[i] = bf < total;
    const int s = bf & (nseq - 1);
    const int rest = bf >> mp.lnseq;
    const int b = rest % nbf;
    const int g = rest / nbf;
    kk[i] = b & (p - 1);
    addr[i] = g * mp.gstride + s;   // base of the sequence
    if (on[i]) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C t;
        if (ZIN && 2 * r >= R) {          // element b + r N / R >= N / 2
          t.x = 0; t.y = 0;
        } else {
          t = buf[il_at<PIN>(addr[i] + ((b + r * nbf) << mp.lnseq))];
        }
        if (INV) t.y = -t.y;
        v[i * R + r] = t;
      }
    }
    // output position of element r: (b - k) R + k + r p
    addr[i] += ((b - kk[i]) * R + kk[i]) << mp.lnseq;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (!on[i]) continue;
    C *u = v + i * R;
    const int k = kk[i];
    if (k != 0) {
      // this pass's table: entry (r - 1) p + k is exp(-2 pi i r k / (p R)); butterflies
      // of neighbouring k read neighbouring entries
#pragma unroll
      for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tw[TOFF + (r - 1) * p + k]);
    }
    dft_r<C, R>(u);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (HALFOUT && 2 * r >= R) continue;   // last pass: output k + r N / R >= N / 2
      C t = u[r];
      if (INV) t.y = -t.y;
      buf[il_at<POUT>(addr[i] + ((r * p) << mp.lnseq))] = t;
    }
  }
  __syncthreads();
}

// Compile-time pass schedule for N = 2^LOGN: radix 32 (V >= 32) or 16 while
// possible, then the remaining factor; the passes are straight-line code so every pass's register
// arrays have their own short lifetime.
template <typename C, int V, bool INV, int N, int P, bool ZIN, bool HALFOUT, bool PIN = false, int TOFF = 0>
__device__ __forceinline__ void fft_passes(C *buf, IlMap mp, const C *__restrict__ tw) {
  if constexpr (P < N) {
    constexpr int REM = N / P;
    constexpr int RMAX = V >= 32 ? 32 : 16;      // radix 32 when a thread holds 32 values
    constexpr int R = REM >= RMAX ? RMAX : REM;
    constexpr bool POUT = P == 1 && P * R < N;   // the first pass writes padded unless it is the last
    il_pass<C, R, V, INV, ZIN && P == 1, HALFOUT && P * R == N, PIN, POUT, TOFF>(buf, N, P, mp, tw);
    fft_passes<C, V, INV, N, P * R, ZIN, HALFOUT, POUT, TOFF + (P > 1 ? (R - 1) * P : 0)>(buf, mp, tw);
  }
}

// Twiddle tables of the passes of a length-N transform, one after the other in
// the order of the passes (the first pass needs none): for a pass after p
// elements with radix R, entry (r - 1) p + k (r = 1..R-1, k < p) holds
// exp(-2 pi i r k / (p R)), taken from the 4096-entry table tw4096.  Together
// they take at most N entries.
template <typename C, int V, int N, int P, int TOFF>
__device__ __forceinline__ void il_build_tw(C *tab, const C *__restrict__ tw4096, int shift) {
  if constexpr (P < N) {
    constexpr int REM = N / P;
    constexpr int RMAX = V >= 32 ? 32 : 16;
    constexpr int R = REM >= RMAX ? RMAX : REM;
    if constexpr (P > 1) {
      constexpr int Q = N / (P * R);
      for (int t = threadIdx.x; t < (R - 1) * P; t += blockDim.x) {
        const int r = 1 + t / P, k = t % P;      // P is a power of two
        tab[TOFF + t] = tw4096[((r * k * Q) & (N - 1)) << shift];
      }
    }
    il_build_tw<C, V, N, P * R, TOFF + (P > 1 ? (R - 1) * P : 0)>(tab, tw4096, shift);
  }
}

template <typename C, int V>
__device__ __forceinline__ void il_twiddles(C *tab, const C *__restrict__ tw4096, int logN) {
  const int sh = 12 - logN;
  switch (logN) {
    case 1: il_build_tw<C, V, 2, 1, 0>(tab, tw4096, sh); break;
    case 2: il_build_tw<C, V, 4, 1, 0>(tab, tw4096, sh); break;
    case 3: il_build_tw<C, V, 8, 1, 0>(tab, tw4096, sh); break;
    case 4: il_build_tw<C, V, 16, 1, 0>(tab, tw4096, sh); break;
    case 5: il_build_tw<C, V, 32, 1, 0>(tab, tw4096, sh); break;
    case 6: il_build_tw<C, V, 64, 1, 0>(tab, tw4096, sh); break;
    case 7: il_build_tw<C, V, 128, 1, 0>(tab, tw4096, sh); break;
    case 8: il_build_tw<C, V, 256, 1, 0>(tab, tw4096, sh); break;
    case 9: il_build_tw<C, V, 512, 1, 0>(tab, tw4096, sh); break;
    case 10: il_build_tw<C, V, 1024, 1, 0>(tab, tw4096, sh); break;
    case 11: il_build_tw<C, V, 2048, 1, 0>(tab, tw4096, sh); break;
    case 12: il_build_tw<C, V, 4096, 1, 0>(tab, tw4096, sh); break;
    default: break;
  }
}

// Full transform (forward or unnormalized inverse), 2 <= N <= 4096.
// blockDim.x * V must cover ngroups * nseq * N elements; tw holds the pass
// tables of il_twiddles (typically in shared memory).  ZIN: the upper half of
// every input sequence is zero (zero padding) and is never read; HALFOUT: only
// the lower half of every output is written back.
template <typename C, int V, bool INV, bool ZIN = false, bool HALFOUT = false>
__device__ __forceinline__ void fft_il(C *buf, int logN, IlMap mp, const C *__restrict__ tw) {
  switch (logN) {
    case 1: fft_passes<C, V, INV, 2, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 2: fft_passes<C, V, INV, 4, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 3: fft_passes<C, V, INV, 8, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 4: fft_passes<C, V, INV, 16, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 5: fft_passes<C, V, INV, 32, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 6: fft_passes<C, V, INV, 64, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 7: fft_passes<C, V, INV, 128, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 8: fft_passes<C, V, INV, 256, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 9: fft_passes<C, V, INV, 512, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 10: fft_passes<C, V, INV, 1024, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 11: fft_passes<C, V, INV, 2048, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    case 12: fft_passes<C, V, INV, 4096, 1, ZIN, HALFOUT>(buf, mp, tw); break;
    default: break;
  }
}

}  // namespace mmc
