// Shared-memory complex FFTs for the demag convolution (Sec. III, Eq. 14).
//
// Stockham autosort formulation, radix-8 passes followed by one radix-4 or
// radix-2 pass for the remaining factor.  A sequence of length N (power of two,
// 2 <= N <= 4096) is handled by G = max(N/8, 1) threads; every thread keeps the
// 8 values of its butterflies in registers for one pass, so a pass is one
// shared-memory read and one write of the sequence (two __syncthreads).
// Twiddles come from a device table tw[t] = exp(-2 pi i t / 4096) built on the
// host in FP64.
#pragma once

#include <cuda_runtime.h>

namespace mmc {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// multiply by -i
template <typename C> __device__ __forceinline__ C cmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// FP32 complex sums as one packed two-lane instruction each (Blackwell's
// FADD2: both components in one issue, rounded like two FADDs)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// in-register forward DFTs
template <typename C> __device__ __forceinline__ void dft2(C &a, C &b) {
  C t = a; a = cadd(t, b); b = csub(t, b);
}
template <typename C> __device__ __forceinline__ void dft4(C *v) {
  C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  C b0 = cadd(v[1], v[3]), b1 = cmi(csub(v[1], v[3]));
  v[0] = cadd(a0, b0); v[2] = csub(a0, b0);
  v[1] = cadd(a1, b1); v[3] = csub(a1, b1);
}
// FP32: the sums packed; the two outputs that take -i (v1 - v3) add its
// swapped components, which stays two scalar adds each
__device__ __forceinline__ void dft4(float2 *v) {
  const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  const float2 b0 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  v[1] = make_float2(a1.x + d.y, a1.y - d.x);
  v[3] = make_float2(a1.x - d.y, a1.y + d.x);
}
template <typename C> __device__ __forceinline__ void dft8(C *v) {
  using R = decltype(v[0].x);
  const R h = (R)0.70710678118654752440;
  C e[4] = {v[0], v[2], v[4], v[6]};
  C o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e);
  dft4(o);
  // o[k] *= exp(-2 pi i k / 8)
  C o1; o1.x = h * (o[1].x + o[1].y); o1.y = h * (o[1].y - o[1].x);
  C o2 = cmi(o[2]);
  C o3; o3.x = h * (o[3].y - o[3].x); o3.y = -h * (o[3].x + o[3].y);
  v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}
// FP32: as above with the packed sums; the -i rotation of o[2] stays scalar
__device__ __forceinline__ void dft8(float2 *v) {
  const float h = 0.70710678118654752440f;
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e);
  dft4(o);
  const float2 o1 = make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
  const float2 o3 = make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
  v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
  v[2] = make_float2(e[2].x + o[2].y, e[2].y - o[2].x);
  v[6] = make_float2(e[2].x - o[2].y, e[2].y + o[2].x);
  v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}

// Addressing of a family of sequences inside shared memory: sequence f starts
// at (f / inner) * so + (f % inner) * si; element e of it is at start + e * se.
struct SeqMap {
  int inner, so, si, se;
  __device__ __forceinline__ int start(int f) const { return (f / inner) * so + (f % inner) * si; }
};

// One Stockham pass of radix R (8, 4 or 2) after p elements: every thread
// loads its `per` butterflies (per <= 8 / R), all threads synchronize, then
// twiddle, transform and store them.  R is a compile-time constant so that the
// butterflies' values stay in registers.
template <typename C, int R>
__device__ __forceinline__ void fft_smem_pass(C *buf, int N, int p, int G, int g, int st, int se, bool active,
                                              int twshift, const C *__restrict__ tw) {
  const int nbf = N / R;                       // butterflies in this pass
  const int per = nbf / G;                     // butterflies per thread (1, 2 or 4)
  C v[8];
  if (active) {
#pragma unroll
    for (int t = 0; t < 8 / R; ++t) {
      if (t >= per) break;
      const int b = g + t * G;
#pragma unroll
      for (int r = 0; r < R; ++r) v[t * R + r] = buf[st + (b + r * nbf) * se];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int t = 0; t < 8 / R; ++t) {
      if (t >= per) break;
      const int b = g + t * G;
      const int k = b & (p - 1);
      C *u = v + t * R;
      if (k != 0) {
        // twiddle exp(-2 pi i r k / (p R)): table index r * k * N / (p R)
        const int step = (k * (N / (p * R))) << twshift;
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tw[(r * step) & 4095]);
      }
      if (R == 8) dft8(u);
      else if (R == 4) dft4(u);
      else dft2(u[0], u[1]);
      const int j = (b - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[st + (j + r * p) * se] = u[r];
    }
  }
  __syncthreads();
}

// Forward (inverse = false) or inverse (unnormalized) FFT of nseq sequences of
// length N = 2^logN in place in shared memory.  Every thread of the block must
// call it.  The inverse is computed as conj(FFT(conj(x))).
template <typename C>
__device__ void fft_smem(C *buf, int logN, int nseq, SeqMap map, const C *__restrict__ tw,
                         bool inverse) {
  const int N = 1 << logN;
  const int G = N >= 8 ? N >> 3 : 1;           // threads per sequence
  const int groups = blockDim.x / G;
  const int g = threadIdx.x % G;
  const int grp = threadIdx.x / G;
  const int twshift = 12 - logN;               // table length 4096 = 2^12
  for (int base = 0; base < nseq; base += groups) {
    const int f = base + grp;
    const bool active = (grp < groups) && (f < nseq);
    const int st = active ? map.start(f) : 0;
    if (inverse && active)
      for (int e = g; e < N; e += G) {
        C &x = buf[st + e * map.se];
        x.y = -x.y;
      }
    __syncthreads();
    int p = 1;
    while (p < N) {
      const int rem = N / p;
      if (rem >= 8) {
        fft_smem_pass<C, 8>(buf, N, p, G, g, st, map.se, active, twshift, tw);
        p *= 8;
      } else if (rem == 4) {
        fft_smem_pass<C, 4>(buf, N, p, G, g, st, map.se, active, twshift, tw);
        p *= 4;
      } else {
        fft_smem_pass<C, 2>(buf, N, p, G, g, st, map.se, active, twshift, tw);
        p *= 2;
      }
    }
    if (inverse && active)
      for (int e = g; e < N; e += G) {
        C &x = buf[st + e * map.se];
        x.y = -x.y;
      }
    __syncthreads();
  }
}

}  // namespace mmc
