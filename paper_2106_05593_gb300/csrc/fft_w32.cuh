// Warp-resident 1024-point FFTs for the 2D demag convolution (Sec. III, Eq. 14).
//
// One warp owns one sequence z of length 1024 as a 32 x 32 split, n = 32 n1 + n2
// and k = k1 + 32 k2:
//   1. lane n2 holds z[32 n1 + n2] for n1 = 0..31 and takes the 32-point DFT
//      over n1 in registers;
//   2. it multiplies output k1 by exp(-2 pi i n2 k1 / 1024);
//   3. the warp transposes the 32 x 32 block through shared memory, so that
//      lane k1 holds the values of every n2;
//   4. lane k1 takes the 32-point DFT over n2 and ends with Z[k1 + 32 k2],
//      k2 = 0..31.
// The inverse runs the same steps with conjugated roots on the other index
// order (lane k1 starts with Z[k1 + 32 k2] and lane n' ends with
// z[n' + 32 n''], unnormalized).  A transform is one shared-memory round trip
// (the transpose) and no block barrier.  The transpose buffer of a warp is
// 32 x 33 complex values (row pitch 33 keeps both access patterns free of bank
// conflicts).  The twiddles of step 2 come from a 32 x 32 table in global
// memory laid out so that the 32 lanes read 32 consecutive entries.
#pragma once

#include "fft_il.cuh"

namespace mmc {

constexpr int kW32N = 1024;
constexpr int kW32Pitch = 33;                       // transpose row pitch (complex values)
constexpr int kW32Buf = 32 * kW32Pitch;             // complex values per warp buffer

// forward 32-point DFT whose inputs 16..31 are zero (zero padding): the first
// radix-4 step of the 4 x 8 split (n = 8 n1 + n2, k = k1 + 4 k2) sees two
// non-zero inputs per butterfly; x[16..31] are not read
__device__ __forceinline__ void dft32_lo16(float2 *x) {
  float2 a[32];
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2) {
    const float2 t0 = x[n2], t1 = x[8 + n2];
    float2 o[4];
    o[0] = cadd(t0, t1);
    o[1] = make_float2(t0.x + t1.y, t0.y - t1.x);      // t0 - i t1
    o[2] = csub(t0, t1);
    o[3] = make_float2(t0.x - t1.y, t0.y + t1.x);      // t0 + i t1
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[4 * n2 + k1] = (n2 * k1) ? cmul_w32(o[k1], n2 * k1) : o[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 t[8] = {a[k1], a[4 + k1], a[8 + k1], a[12 + k1], a[16 + k1], a[20 + k1], a[24 + k1], a[28 + k1]};
    dft8(t);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) x[k1 + 4 * k2] = t[k2];
  }
}

// inverse (unnormalized) 32-point DFT: conj(DFT(conj(x)))
__device__ __forceinline__ void idft32(float2 *x) {
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i].y = -x[i].y;
  dft32(x);
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i].y = -x[i].y;
}

// steps 2-4 of the forward transform: v[k1] (this lane's n2 = lane) times the
// twiddle, the transpose through buf (this warp's kW32Buf values), and the DFT
// over n2; on return v[k2] = Z[lane + 32 k2].  buf is free again on return.
__device__ __forceinline__ void w32_fwd_tail(float2 *v, float2 *buf, const float2 *__restrict__ tw, int lane) {
#pragma unroll
  for (int k1 = 1; k1 < 32; ++k1) v[k1] = cmul(v[k1], __ldg(tw + k1 * 32 + lane));
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) buf[k1 * kW32Pitch + lane] = v[k1];
  __syncwarp();
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) v[n2] = buf[lane * kW32Pitch + n2];
  __syncwarp();
  dft32(v);
}

// the inverse transform of v[k2] = Z[lane + 32 k2]; on return v[n''] =
// z[lane + 32 n''] (unnormalized), of which the first `nout` are used by the
// caller (the compiler drops the work of the others)
__device__ __forceinline__ void w32_inv(float2 *v, float2 *buf, const float2 *__restrict__ tw, int lane) {
  idft32(v);                                           // over k2: v[n'] for k1 = lane
#pragma unroll
  for (int n = 1; n < 32; ++n) v[n] = cmul(v[n], cconj(__ldg(tw + n * 32 + lane)));
#pragma unroll
  for (int n = 0; n < 32; ++n) buf[n * kW32Pitch + lane] = v[n];
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) v[k1] = buf[lane * kW32Pitch + k1];
  __syncwarp();
  idft32(v);                                           // over k1: v[n''] for n' = lane
}

}  // namespace mmc
