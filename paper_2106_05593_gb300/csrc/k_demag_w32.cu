// FP32 2D demag convolution (Sec. III, Eq. 14) for chains whose padded grid
// is 1024 x 1024, on warp-resident 1024-point transforms (fft_w32.cuh).
//
// Spectrum layout (per chain, at ChainDev::s_off; R4 = rows rounded up to 4,
// Sx = 520 the row stride of every 1024-point grid): component c, row y and
// column kx at
//   c R4 Sx + (y / 4) 4 Sx + 4 kx + y % 4,
// i.e. tiles of four rows stored column by column.  The forward row kernel
// writes one whole tile per component (contiguous); the column kernel reads and
// writes a column as 32-byte runs of four rows.
//
// Three kernels, as in the interleaved path:
//   k_w32_rows_fwd  one block per tile of 4 rows (6 warps): Ms0 m of two rows
//                   packed per complex sequence, (x + i y of each row, z of both
//                   rows), forward transforms, Hermitian split to the half
//                   spectra kx <= 512, the tile written out.
//   k_w32_cols      one block per column kx (3 warps, one per component):
//                   forward column transforms (rows >= ny are zero padding),
//                   H = -N M with the tensor spectra, inverse transforms, rows
//                   y < ny written back.
//   k_w32_rows_inv  one block per tile: the packed sequences z = a + i b built
//                   from the half spectra, inverse transforms, the crop x < nx,
//                   and the sweep's field zee (B + mu0 H) in the split layout.
#include "demag_args.cuh"
#include "fft_w32.cuh"
#include "tma.cuh"

namespace mmc {

struct W32Args {
  const ChainDev *chains;
  const int *blk_chain;
  const long long *blk_first;
  const float4 *m;
  const float4 *tab;
  const float *ms;
  float2 *S;
  const float *const *nhatT;      // per tensor set: [comp][kx][kyq], comps xx yy zz xy, 513 x 513
  const float2 *tw;               // tw[k1 * 32 + t] = exp(-2 pi i t k1 / 1024)
  float4 *heff;
  double *Hd;
  int Hd_chain;
  int *err;                       // device error word (a wait for the tensor copy that gave up)
};

constexpr int kW32Half = 513;           // kx = 0..512
constexpr int kW32TPitch = kW32TensorPitch;                    // tensor row (kyq) pitch, 16-byte multiple
constexpr long long kW32TQ = (long long)kW32Half * kW32TPitch; // one tensor component
constexpr int kW32Sx = 520;             // spectrum row stride of a 1024-point grid (complex values)
constexpr int kW32Tile = 4 * kW32Sx;    // one tile of four rows
constexpr int kW32TilePitch = 524;      // smem row pitch of the row kernels' tiles
constexpr unsigned kW32Polls = 1u << 22;

__device__ __forceinline__ long long w32_at(const ChainDev &ch, int comp, int y, int kx) {
  const long long R4 = (long long)((ch.nrows + 3) & ~3);
  return ch.s_off + (long long)comp * R4 * kW32Sx + (long long)(y >> 2) * kW32Tile + 4LL * kx + (y & 3);
}

__global__ void __launch_bounds__(192, 3) k_w32_rows_fwd(W32Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  const int c = A.blk_chain[blockIdx.x];
  const ChainDev &ch = A.chains[c];
  const int tile = (int)(blockIdx.x - A.blk_first[c]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = w / 3, q = w - 3 * p;                  // pair in the tile, sequence kind
  const int r0 = 4 * tile + 2 * p, r1 = r0 + 1;
  const int nx = ch.nx, ny = ch.ny;
  float2 *buf = sm + w * kW32Buf;

  // z = Mx + i My of row r0 (q = 0) or r1 (q = 1), or Mz(r0) + i Mz(r1) (q = 2).
  // Cell x = 32 n1 + lane of row r is in colour (lane + r) & 1 at slot
  // 16 n1 + lane / 2 (one-cell-thick chain: row r = j)
  const long long S = (long long)ch.nrows * ch.hx;
  const bool pc = ch.ms_off >= 0;
  const float Msu = (float)ch.Ms0d;
  const int ra = q == 1 ? r1 : r0;                     // the row of x + i y, or of Mz (q = 2)
  const long long oa = (long long)((lane + ra) & 1) * S + (long long)ra * ch.hx + (lane >> 1);
  const long long ob = (long long)((lane + r1) & 1) * S + (long long)r1 * ch.hx + (lane >> 1);
  const float4 *ma = A.m + ch.m_off + oa, *mb = A.m + ch.m_off + ob;
  const bool ha = ra < ny, hb = q == 2 && r1 < ny;
  float2 v[32];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) {
    const bool in = 32 * n1 + lane < nx;
    float2 z = make_float2(0.f, 0.f);
    if (in && ha) {
      const float4 t = ma[16 * n1];
      const float Ms = pc ? A.ms[ch.ms_off + oa + 16 * n1] : Msu;
      z = q == 2 ? make_float2(Ms * t.z, 0.f) : make_float2(Ms * t.x, Ms * t.y);
    }
    if (in && hb) {
      const float4 t = mb[16 * n1];
      const float Ms = pc ? A.ms[ch.ms_off + ob + 16 * n1] : Msu;
      z.y = Ms * t.z;
    }
    v[n1] = z;
  }
  dft32_lo16(v);
  w32_fwd_tail(v, buf, A.tw, lane);                    // v[k2] = Z[lane + 32 k2]

  // Hermitian split: the half spectra of the two real sequences of z,
  // X[k] = (Z[k] + conj Z[N-k]) / 2 and Y[k] = (Z[k] - conj Z[N-k]) / (2i)
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) buf[lane + 32 * k2] = v[k2];
  __syncwarp();
  float2 X[17], Y[17];
#pragma unroll
  for (int k2 = 0; k2 < 17; ++k2) {
    if (k2 == 16 && lane != 0) break;                  // k = 512 belongs to lane 0
    const int k = lane + 32 * k2;
    const float2 Z = v[k2], Zm = buf[(kW32N - k) & (kW32N - 1)];
    X[k2] = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
    Y[k2] = make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));
  }
  __syncthreads();                                     // every warp done with its buffer
  // output tile [comp][row][kx] in shared memory (aliases the warp buffers; row
  // pitch kW32TilePitch keeps the stores and the gather below free of bank conflicts)
  const int cA = q == 2 ? 2 : 0, cB = q == 2 ? 2 : 1;
  const int rA = q == 1 ? 2 * p + 1 : 2 * p, rB = q == 0 ? 2 * p : 2 * p + 1;
#pragma unroll
  for (int k2 = 0; k2 < 17; ++k2) {
    if (k2 == 16 && lane != 0) break;
    const int k = lane + 32 * k2;
    sm[(cA * 4 + rA) * kW32TilePitch + k] = X[k2];
    sm[(cB * 4 + rB) * kW32TilePitch + k] = Y[k2];
  }
  __syncthreads();
  // the tile of every component is contiguous in global memory: [kx][4 rows],
  // written as float4 pairs (rows 2h, 2h + 1 of one kx)
  constexpr int per = kW32Half * 2;                    // float4 per component
  for (int i = threadIdx.x; i < 3 * per; i += blockDim.x) {
    const int comp = i / per, o = i - comp * per;
    const int kx = o >> 1, h = o & 1;
    const float2 a = sm[(comp * 4 + 2 * h) * kW32TilePitch + kx];
    const float2 b = sm[(comp * 4 + 2 * h + 1) * kW32TilePitch + kx];
    float4 *dst = reinterpret_cast<float4 *>(A.S + w32_at(ch, comp, 4 * tile, 0));
    dst[o] = make_float4(a.x, a.y, b.x, b.y);
  }
}

__global__ void __launch_bounds__(96, 5) k_w32_cols(W32Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  float *tn = reinterpret_cast<float *>(sm + 3 * kW32Buf);   // this column's tensor, [4][kW32TPitch]
  __shared__ uint64_t tbar;
  const int c = A.blk_chain[blockIdx.x];
  const ChainDev &ch = A.chains[c];
  const int kx = (int)(blockIdx.x - A.blk_first[c]);
  const int lane = threadIdx.x & 31, comp = threadIdx.x >> 5;
  const int ny = ch.ny;
  float2 *buf = sm + comp * kW32Buf;
  // the column's four tensor components come in by bulk copy while the
  // forward transforms run
  if (threadIdx.x == 0) {
    mbar_init(&tbar, 1);
    mbar_init_fence();
    const float *src = A.nhatT[ch.spec] + (long long)kx * kW32TPitch;
    mbar_arrive_expect_tx(&tbar, 4u * kW32TPitch * 4u);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      bulk_g2s(tn + t * kW32TPitch, src + (long long)t * kW32TQ, kW32TPitch * 4u, &tbar);
  }
  // column kx of component comp: row y = 32 n1 + lane is in tile 8 n1 + lane / 4
  const long long R4 = (long long)((ch.nrows + 3) & ~3);
  float2 *col = A.S + ch.s_off + (long long)comp * R4 * kW32Sx + (long long)(lane >> 2) * kW32Tile + 4 * kx + (lane & 3);

  float2 v[32];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1)
    v[n1] = 32 * n1 + lane < ny ? col[(long long)n1 * 8 * kW32Tile] : make_float2(0.f, 0.f);
  dft32_lo16(v);
  w32_fwd_tail(v, buf, A.tw, lane);                    // v[k2] = M^_comp(kx, lane + 32 k2)

  // H^ = -N^ M^: the x and y warps exchange their spectra
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) buf[lane + 32 * k2] = v[k2];
  __syncthreads();
  if (!mbar_wait(&tbar, 0u, kW32Polls)) {
    // MMC_ERR_TIMEOUT; this column's field is left as it was.  The copy may
    // still be in flight: give it a fixed time (about a millisecond) to land
    // before the block's shared memory is released.
    if (threadIdx.x == 0) atomicExch(A.err, -3);
    const long long t0 = clock64();
    while (clock64() - t0 < (1LL << 21)) {
    }
    return;
  }
  if (comp < 2) {
    const float2 *other = sm + (1 - comp) * kW32Buf;
    const float *Nd = tn + comp * kW32TPitch;          // xx (x warp) or yy (y warp)
    const float *Nxy = tn + 3 * kW32TPitch;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int ky = lane + 32 * k2;
      const int kyq = ky <= 512 ? ky : kW32N - ky;
      const float nd = Nd[kyq];
      const float nxy = ky <= 512 ? Nxy[kyq] : -Nxy[kyq];
      const float2 o = other[lane + 32 * k2];
      v[k2] = make_float2(-(nd * v[k2].x + nxy * o.x), -(nd * v[k2].y + nxy * o.y));
    }
  } else {
    const float *Nzz = tn + 2 * kW32TPitch;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int ky = lane + 32 * k2;
      const float nz = Nzz[ky <= 512 ? ky : kW32N - ky];
      v[k2] = make_float2(-nz * v[k2].x, -nz * v[k2].y);
    }
  }
  __syncthreads();                                     // the other warp has read this buffer
  w32_inv(v, buf, A.tw, lane);                         // v[n''] = H_comp(kx, row lane + 32 n'')
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2)
    if (lane + 32 * n2 < ny) col[(long long)n2 * 8 * kW32Tile] = v[n2];
}

__global__ void __launch_bounds__(192, 3) k_w32_rows_inv(W32Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  const int c = A.blk_chain[blockIdx.x];
  const ChainDev &ch = A.chains[c];
  const int tile = (int)(blockIdx.x - A.blk_first[c]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = w / 3, q = w - 3 * p;
  const int nx = ch.nx, ny = ch.ny;

  // the tile's half spectra, transposed to [comp][row][kx] (pitch kW32TilePitch)
  {
    constexpr int per = kW32Half * 2;                  // float4 (two rows of one kx) per component
    for (int i = threadIdx.x; i < 3 * per; i += blockDim.x) {
      const int comp = i / per, o = i - comp * per;
      const float4 t = reinterpret_cast<const float4 *>(A.S + w32_at(ch, comp, 4 * tile, 0))[o];
      const int kx = o >> 1, r = 2 * (o & 1);
      sm[(comp * 4 + r) * kW32TilePitch + kx] = make_float2(t.x, t.y);
      sm[(comp * 4 + r + 1) * kW32TilePitch + kx] = make_float2(t.z, t.w);
    }
  }
  __syncthreads();
  // z = a + i b of two half spectra: z[k] = a[k] + i b[k] and z[N - k] = conj a[k]
  // + i conj b[k] (real parts only at k = 0 and N/2)
  const int cA = q == 2 ? 2 : 0, cB = q == 2 ? 2 : 1;
  const int rA = q == 1 ? 2 * p + 1 : 2 * p, rB = q == 0 ? 2 * p : 2 * p + 1;
  const float2 *ta = sm + (cA * 4 + rA) * kW32TilePitch;
  const float2 *tb = sm + (cB * 4 + rB) * kW32TilePitch;
  float2 v[32];
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    const int k = lane + 32 * k2;
    if (k2 < 16) {
      const float2 a = ta[k], b = tb[k];
      v[k2] = k == 0 ? make_float2(a.x, b.x) : make_float2(a.x - b.y, a.y + b.x);
    } else {
      const int km = kW32N - k;                        // 1..512
      const float2 a = ta[km], b = tb[km];
      v[k2] = km == 512 ? make_float2(a.x, b.x) : make_float2(a.x + b.y, b.x - a.y);
    }
  }
  __syncthreads();                                     // the tile is read; its space becomes warp buffers
  w32_inv(v, sm + w * kW32Buf, A.tw, lane);            // v[n''] = z[lane + 32 n''] (unnormalized)
  __syncthreads();                                     // warp buffers free: reuse as the field tile
  // field tile [comp][row][x] (floats, A/m) of the 4 rows
  float *ft = reinterpret_cast<float *>(sm);
  const float scale = 1.f / ((float)kW32N * (float)kW32N);
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) {
    const int x = lane + 32 * n2;
    ft[(cA * 4 + rA) * 512 + x] = v[n2].x * scale;
    ft[(cB * 4 + rB) * 512 + x] = v[n2].y * scale;
  }
  __syncthreads();
  const long long Sl = (long long)ny * ch.hx;
  const bool percell = ch.t_off >= 0;
  const float mu0f = (float)mu0;
  for (int i = threadIdx.x; i < 4 * nx; i += blockDim.x) {
    const int rr = (int)divq((unsigned)i, ch.nx_m, ch.nx_l), x = i - rr * nx;
    const int r = 4 * tile + rr;
    if (r >= ny) break;
    const float Hx = ft[(0 * 4 + rr) * 512 + x], Hy = ft[(1 * 4 + rr) * 512 + x], Hz = ft[(2 * 4 + rr) * 512 + x];
    const int colr = (x + r) & 1;
    const long long li = (long long)colr * Sl + (long long)r * ch.hx + (x >> 1);
    if (A.heff) {
      const float zee = percell ? A.tab[ch.t_off + 2 * Sl + li].x : ch.zee;
      A.heff[ch.h_off + li] = make_float4(zee * (ch.Bx + mu0f * Hx), zee * (ch.By + mu0f * Hy),
                                          zee * (ch.Bz + mu0f * Hz), 0.f);
    }
    if (A.Hd && c == A.Hd_chain) {
      const long long nat = x + (long long)nx * r;
      A.Hd[3 * nat + 0] = (double)Hx;
      A.Hd[3 * nat + 1] = (double)Hy;
      A.Hd[3 * nat + 2] = (double)Hz;
    }
  }
}

constexpr size_t kW32RowsSmem = 6 * kW32Buf * sizeof(float2);
constexpr size_t kW32ColsSmem = 3 * kW32Buf * sizeof(float2) + 4 * kW32TPitch * sizeof(float);
static_assert(kW32RowsSmem >= 12 * kW32TilePitch * sizeof(float2), "output tile fits the warp buffers");
static_assert((3 * kW32Buf * sizeof(float2)) % 16 == 0 && (kW32TPitch * 4) % 16 == 0, "bulk copy alignment");
static_assert(kW32RowsSmem >= 12 * kW32TilePitch * sizeof(float2), "input tile fits the warp buffers");
static_assert(kW32RowsSmem >= 12 * 512 * sizeof(float), "field tile fits the warp buffers");

void launch_w32(const Launch &L, const DemagLaunch &P) {
  W32Args A;
  A.chains = P.chains; A.m = P.m; A.tab = P.tab; A.ms = P.ms;
  A.S = reinterpret_cast<float2 *>(P.spec);
  A.nhatT = reinterpret_cast<const float *const *>(P.nhatT);
  A.tw = reinterpret_cast<const float2 *>(P.tw1024);
  A.heff = P.heff; A.Hd = P.Hd; A.Hd_chain = P.Hd_chain;
  A.err = P.err;
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  if (P.ev) cudaEventRecord(P.ev[0], L.stream);
  k_w32_rows_fwd<<<P.rows_blocks, 192, kW32RowsSmem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[1], L.stream);
  A.blk_chain = P.cols_chain; A.blk_first = P.cols_first;
  k_w32_cols<<<P.cols_blocks, 96, kW32ColsSmem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[2], L.stream);
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  k_w32_rows_inv<<<P.rows_blocks, 192, kW32RowsSmem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[3], L.stream);
  *L.counter += 3;
}

cudaError_t w32_set_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_w32_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kW32RowsSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_w32_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kW32RowsSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_w32_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kW32ColsSmem);
}

}  // namespace mmc
