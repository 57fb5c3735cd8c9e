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
// Twiddles come from the FP64-built table tw[t] = exp(-2 pi i t / 4096).
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

template <typename C, int R> __device__ __forceinline__ void dft_r(C *u) {
  if (R == 16) dft16(u);
  else if (R == 8) dft8(u);
  else if (R == 4) dft4(u);
  else if (R == 2) dft2(u[0], u[1]);
}

struct IlMap {
  int nseq, ngroups, gstride;
};

// one radix-R Stockham pass over all interleaved sequences (p = product of the
// radices already done); V values per thread
template <typename C, int R, int V, bool INV>
__device__ __forceinline__ void il_pass(C *buf, int N, int p, IlMap mp, const C *__restrict__ tw, int twshift) {
  constexpr int NB = V / R;
  const int nbf = N / R;
  const int total = mp.ngroups * nbf * mp.nseq;
  C v[V];
  int addr[NB], kk[NB];
  bool on[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int bf = threadIdx.x + i * blockDim.x;
    on[i] = bf < total;
    const int s = bf % mp.nseq;
    const int rest = bf / mp.nseq;
    const int b = rest % nbf;
    const int g = rest / nbf;
    kk[i] = b & (p - 1);
    addr[i] = g * mp.gstride + s;   // base of the sequence
    if (on[i]) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C t = buf[addr[i] + (b + r * nbf) * mp.nseq];
        if (INV) t.y = -t.y;
        v[i * R + r] = t;
      }
    }
    // output position of element r: (b - k) R + k + r p
    addr[i] += ((b - kk[i]) * R + kk[i]) * mp.nseq;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (!on[i]) continue;
    C *u = v + i * R;
    const int k = kk[i];
    if (k != 0) {
      const int step = (k * (N / (p * R))) << twshift;
#pragma unroll
      for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tw[(r * step) & 4095]);
    }
    dft_r<C, R>(u);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C t = u[r];
      if (INV) t.y = -t.y;
      buf[addr[i] + r * p * mp.nseq] = t;
    }
  }
  __syncthreads();
}

// Compile-time pass schedule for N = 2^LOGN: radix 16 while possible, then the
// remaining factor; the passes are straight-line code so every pass's register
// arrays have their own short lifetime.
template <typename C, int V, bool INV, int N, int P>
__device__ __forceinline__ void fft_passes(C *buf, IlMap mp, const C *__restrict__ tw, int twshift) {
  if constexpr (P < N) {
    constexpr int REM = N / P;
    constexpr int R = REM >= 16 ? 16 : REM;
    il_pass<C, R, V, INV>(buf, N, P, mp, tw, twshift);
    fft_passes<C, V, INV, N, P * R>(buf, mp, tw, twshift);
  }
}

// Full transform (forward or unnormalized inverse), 2 <= N <= 4096.
// blockDim.x * V must cover ngroups * nseq * N elements.
template <typename C, int V, bool INV>
__device__ __forceinline__ void fft_il(C *buf, int logN, IlMap mp, const C *__restrict__ tw) {
  const int twshift = 12 - logN;
  switch (logN) {
    case 1: fft_passes<C, V, INV, 2, 1>(buf, mp, tw, twshift); break;
    case 2: fft_passes<C, V, INV, 4, 1>(buf, mp, tw, twshift); break;
    case 3: fft_passes<C, V, INV, 8, 1>(buf, mp, tw, twshift); break;
    case 4: fft_passes<C, V, INV, 16, 1>(buf, mp, tw, twshift); break;
    case 5: fft_passes<C, V, INV, 32, 1>(buf, mp, tw, twshift); break;
    case 6: fft_passes<C, V, INV, 64, 1>(buf, mp, tw, twshift); break;
    case 7: fft_passes<C, V, INV, 128, 1>(buf, mp, tw, twshift); break;
    case 8: fft_passes<C, V, INV, 256, 1>(buf, mp, tw, twshift); break;
    case 9: fft_passes<C, V, INV, 512, 1>(buf, mp, tw, twshift); break;
    case 10: fft_passes<C, V, INV, 1024, 1>(buf, mp, tw, twshift); break;
    case 11: fft_passes<C, V, INV, 2048, 1>(buf, mp, tw, twshift); break;
    case 12: fft_passes<C, V, INV, 4096, 1>(buf, mp, tw, twshift); break;
    default: break;
  }
}

}  // namespace mmc
