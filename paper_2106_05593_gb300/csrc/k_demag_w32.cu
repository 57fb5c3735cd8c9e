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
#include <cuda.h>

#include "demag_args.cuh"
#include "fft_w32.cuh"
#include "philox.cuh"
#include "tma.cuh"
#include "trial.cuh"

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
  MmcCheck *ck;                   // checked builds: the record (checked.cuh)
  int nchains;                    // entries of the chain table
};

constexpr int kW32Half = 513;           // kx = 0..512
constexpr int kW32TPitch = kW32TensorPitch;                    // tensor row (kyq) pitch, 16-byte multiple
constexpr long long kW32TQ = (long long)kW32Half * kW32TPitch; // one tensor component
constexpr int kW32TilePitch = 524;      // smem row pitch of the row kernels' tiles
constexpr unsigned kW32Polls = 1u << 22;

__device__ __forceinline__ long long w32_at(const ChainDev &ch, int comp, int y, int kx) {
  const long long R4 = (long long)((ch.nrows + 3) & ~3);
  return ch.s_off + (long long)comp * R4 * kW32Sx + (long long)(y >> 2) * kW32Tile + 4LL * kx + (y & 3);
}

// index of float2 pair o (two rows of one kx) of component comp's tile `tile`,
// checked against the chain's spectrum
__device__ __forceinline__ long long w32_tile_pair(const W32Args &A, const ChainDev &ch, int comp, int tile, int o) {
  const long long R4 = (long long)((ch.nrows + 3) & ~3);
  return MMC_CKR(A.ck, w32_at(ch, comp, 4 * tile, 0) + 2LL * o, 2, ch.s_off, ch.s_off + 3 * R4 * kW32Sx,
                 kCkDemagSpectrum);
}

// the block's chain, checked against the chain table
__device__ __forceinline__ int w32_chain_of_block(const W32Args &A) {
  return (int)MMC_CK(A.ck, A.blk_chain[blockIdx.x], 0, A.nchains, kCkDemagBlock);
}

__global__ void __launch_bounds__(192, 3) k_w32_rows_fwd(W32Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  const int c = w32_chain_of_block(A);
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
      const float4 t = ma[MMC_CK(A.ck, 16 * n1, -oa, 2 * S - oa, kCkDemagM)];
      const float Ms = pc ? A.ms[ch.ms_off + MMC_CK(A.ck, oa + 16 * n1, 0, 2 * S, kCkDemagM)] : Msu;
      z = q == 2 ? make_float2(Ms * t.z, 0.f) : make_float2(Ms * t.x, Ms * t.y);
    }
    if (in && hb) {
      const float4 t = mb[MMC_CK(A.ck, 16 * n1, -ob, 2 * S - ob, kCkDemagM)];
      const float Ms = pc ? A.ms[ch.ms_off + MMC_CK(A.ck, ob + 16 * n1, 0, 2 * S, kCkDemagM)] : Msu;
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
    *reinterpret_cast<float4 *>(A.S + w32_tile_pair(A, ch, comp, tile, o)) = make_float4(a.x, a.y, b.x, b.y);
  }
}

// The spectrum seen as a 2D tensor for the column loads (tensor map tmS): a
// row of the tensor is one tile of four rows (kW32Tile complex values = 4160
// floats), so one kx of a tile is 8 consecutive floats; a box of 8 floats x
// kW32ColTiles tiles is one 512-row column of one component.  Boxes of chains
// with fewer rows reach into the next component's tiles (read, not used), and
// past the end of the buffer they read zeros.
constexpr int kW32ColTiles = 128;
constexpr unsigned kW32ColBytes = kW32ColTiles * 32u;
static_assert(kW32ColBytes + 128 <= kW32Buf * sizeof(float2), "a column box fits a warp buffer");

__global__ void __launch_bounds__(96, 5) k_w32_cols(W32Args A, const __grid_constant__ CUtensorMap tmS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  float *tn = reinterpret_cast<float *>(sm + 3 * kW32Buf);   // this column's tensor, [4][kW32TPitch]
  __shared__ uint64_t tbar, cbar[3];
  const int c = w32_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int kx = (int)(blockIdx.x - A.blk_first[c]);
  const int lane = threadIdx.x & 31, comp = threadIdx.x >> 5;
  const int ny = ch.ny;
  float2 *buf = sm + comp * kW32Buf;
  // this warp's column of the spectrum comes in as one box of the tensor map,
  // into the start of the warp's buffer rounded up to 128 bytes
  const long long R4 = (long long)((ch.nrows + 3) & ~3);
  // (an offset from buf, so that the compiler keeps the shared-memory accesses)
  float2 *colbuf = buf + ((128u - (smem_u32(buf) & 127u)) & 127u) / sizeof(float2);
  if (lane == 0) {
    mbar_init(&cbar[comp], 1);
    mbar_init_fence();
    mbar_arrive_expect_tx(&cbar[comp], kW32ColBytes);
    const long long t0 = ch.s_off / kW32Tile;
    const long long tile0 = MMC_CK(A.ck, t0 + (long long)comp * (R4 / 4), t0, t0 + 3 * (R4 / 4), kCkDemagSpectrum);
    tma_load_2d(colbuf, &tmS, 8 * (int)MMC_CK(A.ck, kx, 0, kW32Half, kCkDemagSpectrum), (int)tile0, &cbar[comp]);
  }
  __syncwarp();
  // the column's four tensor components come in by bulk copy while the
  // forward transforms run
  if (threadIdx.x == 0) {
    mbar_init(&tbar, 1);
    mbar_init_fence();
    const float *src = A.nhatT[ch.spec];
    mbar_arrive_expect_tx(&tbar, 4u * kW32TPitch * 4u);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      bulk_g2s(tn + t * kW32TPitch,
               src + MMC_CKR(A.ck, (long long)kx * kW32TPitch + (long long)t * kW32TQ, kW32TPitch, 0, 4 * kW32TQ,
                             kCkDemagTensor),
               kW32TPitch * 4u, &tbar);
  }
  // column kx of component comp: row y = 32 n1 + lane is in tile 8 n1 + lane / 4
  const long long cb = (long long)comp * R4 * kW32Sx + (long long)(lane >> 2) * kW32Tile + 4 * kx + (lane & 3);
  float2 *col = A.S + ch.s_off + cb;
  const long long clo = -cb, chi = 3 * R4 * kW32Sx - cb;   // the chain's spectrum, relative to col

  // in the box, row y is at tile y / 4, element y % 4: float2 index y
  float2 v[32];
  const bool col_ok = mbar_wait(&cbar[comp], 0u, kW32Polls);
  if (!col_ok && lane == 0) atomicExch(A.err, -3);      // MMC_ERR_TIMEOUT; this column's field is wrong
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1)
    v[n1] = col_ok && 32 * n1 + lane < ny ? colbuf[32 * n1 + lane] : make_float2(0.f, 0.f);
  __syncwarp();                                        // the box is read: the buffer takes the transpose
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
    if (lane + 32 * n2 < ny) col[MMC_CK(A.ck, (long long)n2 * 8 * kW32Tile, clo, chi, kCkDemagSpectrum)] = v[n2];
  if (!col_ok) {
    // the box may still land in the block's shared memory: give it a fixed
    // time (about a millisecond) before the block exits
    const long long t0 = clock64();
    while (clock64() - t0 < (1LL << 21)) {
    }
  }
}

__global__ void __launch_bounds__(192, 3) k_w32_rows_inv(W32Args A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  const int c = w32_chain_of_block(A);
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
      const float4 t = *reinterpret_cast<const float4 *>(A.S + w32_tile_pair(A, ch, comp, tile, o));
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
    const long long li = MMC_CK(A.ck, (long long)colr * Sl + (long long)r * ch.hx + (x >> 1), 0, 2 * Sl, kCkDemagField);
    if (A.heff) {
      const float zee = percell ? A.tab[ch.t_off + 2 * Sl + li].x : ch.zee;
      A.heff[ch.h_off + li] = make_float4(zee * (ch.Bx + mu0f * Hx), zee * (ch.By + mu0f * Hy),
                                          zee * (ch.Bz + mu0f * Hz), 0.f);
    }
    if (A.Hd && c == A.Hd_chain) {
      const long long nat = MMC_CK(A.ck, x + (long long)nx * r, 0, (long long)nx * ny, kCkDemagField);
      A.Hd[3 * nat + 0] = (double)Hx;
      A.Hd[3 * nat + 1] = (double)Hy;
      A.Hd[3 * nat + 2] = (double)Hz;
    }
  }
}

// ---------------------------------------------------------------------------
// The black sublattice pass of a tile of four rows fused with the forward row
// transforms of the next iteration's demag update (uniform one-cell-thick
// chains on this path).  Once the black pass of a tile is done its four rows
// are final for the iteration (the red cells were final after the red pass),
// so the block can transform them at once.  The tile's black rows, the red rows
// r0 - 1 .. r0 + 4 (halo rows wrapped on periodic y axes, left out at open
// edges) and the black h_eff rows come into shared memory by bulk copy; the
// black pass runs there (the moves of the per-block pass, cell for cell) and
// writes its accepted moves to the tile and to the state; the transforms then
// read every M value from the tiles.
constexpr int kFusedHx = 256;                          // largest hx on this path (nx <= 512)
constexpr int kFusedThreads = 192;
constexpr size_t kFusedSmem = (size_t)14 * kFusedHx * sizeof(float4);
static_assert(kFusedSmem >= 6 * kW32Buf * sizeof(float2), "the tiles cover the warp buffers");

struct FusedArgs {
  W32Args W;
  float4 *m;                    // the state (written by the pass)
  ChainState *st;
  const float4 *heff;           // the sweep's field, split layout
  const unsigned *sweep_base;
  unsigned sweep_off;
  unsigned rk[20];              // Philox round keys
  unsigned max_polls;
};

__global__ void __launch_bounds__(kFusedThreads, 3) k_w32_black_rows_fwd(FusedArgs F) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  float4 *tb = reinterpret_cast<float4 *>(smem_raw);  // black rows r0 .. r0 + nr - 1, pitch hx
  float4 *tr = tb + 4 * kFusedHx;                      // red rows r0 - 1 .. r0 + nr, pitch hx
  float4 *th = tr + 6 * kFusedHx;                      // black h_eff rows r0 .. r0 + nr - 1
  __shared__ uint64_t bar;
  __shared__ float4 skv[kChainKVec];
  __shared__ unsigned wacc[kFusedThreads / 32], watt[kFusedThreads / 32];
  const W32Args &A = F.W;
  const int c = w32_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int tile = (int)(blockIdx.x - A.blk_first[c]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = ch.nx, ny = ch.ny, hx = ch.hx;
  const int r0 = 4 * tile, nr = min(4, ny - r0);
  const long long S = (long long)ch.nrows * hx;
  const float4 *mred = A.m + ch.m_off;
  float4 *mblk = F.m + ch.m_off + S;
  if (threadIdx.x < kChainKVec) skv[threadIdx.x] = __ldg(reinterpret_cast<const float4 *>(A.chains + c) + threadIdx.x);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    const bool pby = (ch.pbc & 2) != 0;
    const int rb = r0 > 0 ? r0 - 1 : (pby ? ny - 1 : -1);
    const int ra = r0 + nr < ny ? r0 + nr : (pby ? 0 : -1);
    const unsigned row_b = (unsigned)hx * 16u;
    mbar_arrive_expect_tx(&bar, 3u * (unsigned)nr * row_b + (rb >= 0 ? row_b : 0u) + (ra >= 0 ? row_b : 0u));
    // row offsets within one colour of the chain (S slots)
    const long long o0 = MMC_CKR(A.ck, (long long)r0 * hx, (long long)nr * hx, 0, S, kCkFusedCopy);
    bulk_g2s(tb, mblk + o0, (unsigned)nr * row_b, &bar);
    bulk_g2s(tr + hx, mred + o0, (unsigned)nr * row_b, &bar);
    if (rb >= 0) bulk_g2s(tr, mred + MMC_CKR(A.ck, (long long)rb * hx, hx, 0, S, kCkFusedCopy), row_b, &bar);
    if (ra >= 0)
      bulk_g2s(tr + (long long)(nr + 1) * hx, mred + MMC_CKR(A.ck, (long long)ra * hx, hx, 0, S, kCkFusedCopy), row_b,
               &bar);
    bulk_g2s(th, F.heff + ch.h_off + S + o0, (unsigned)nr * row_b, &bar);
  }
  __syncthreads();
  const ChainK K = load_chain_vec(skv);
  if (!mbar_wait(&bar, 0u, F.max_polls)) {
    if (threadIdx.x == 0) atomicExch(A.err, -3);      // MMC_ERR_TIMEOUT: this tile is left as it was
    const long long t0 = clock64();
    while (clock64() - t0 < (1LL << 21)) {
    }
    return;
  }

  // 1. the black pass (colour 1) on the tile's cells
  const unsigned sweep = *F.sweep_base + F.sweep_off;
  const float omc = F.st[c].omc;
  const int pbc = K.pbc & 3, flags = K.flags;
  const unsigned nslots = (unsigned)(nr * hx);
  unsigned na = 0, nv = 0;
#pragma unroll 1
  for (int e0 = 0; e0 < 6; e0 += 2) {                  // 4 rows x 256 slots over 192 threads
    bool valid[2];
    unsigned ql[2], cellid[2];
    float4 a[2], h[2], nb[2][4];
    float pres[2][4];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const unsigned q = threadIdx.x + (unsigned)((e0 + e) * kFusedThreads);
      bool ok = q < nslots;
      const int rl = ok ? (int)divq(q, K.hx_m, K.hx_l) : 0;
      const int sl = (int)(q - (unsigned)rl * (unsigned)hx);
      const int j = r0 + rl;
      const int pp = (j + 1) & 1;
      const int i = 2 * sl + pp;
      ok = ok && (i < nx);
      valid[e] = ok;
      ql[e] = q;
      cellid[e] = (unsigned)i + (unsigned)nx * (unsigned)j;
      if (ok) {
        a[e] = tb[q];
        const float4 *O = tr + (rl + 1) * hx + sl;
        const bool hl = i > 0 || (pbc & 1), hr = i < nx - 1 || (pbc & 1);
        const bool hu = j > 0 || (pbc & 2), hd = j < ny - 1 || (pbc & 2);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        nb[e][0] = hl ? O[i > 0 ? pp - 1 : hx - 1] : z4;
        nb[e][1] = hr ? O[i < nx - 1 ? pp : 1 - hx] : z4;
        nb[e][2] = hu ? O[-hx] : z4;
        nb[e][3] = hd ? O[hx] : z4;
        pres[e][0] = hl ? 1.f : 0.f;
        pres[e][1] = hr ? 1.f : 0.f;
        pres[e][2] = hu ? 1.f : 0.f;
        pres[e][3] = hd ? 1.f : 0.f;
        if (flags & F_GRAIN) {
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (nb[e][b].w != a[e].w) pres[e][b] *= K.gscale;
        }
        h[e] = th[q];
      }
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int acc = 0;
      if (valid[e]) {
        const float wv[4] = {K.wx * pres[e][0], K.wx * pres[e][1], K.wy * pres[e][2], K.wy * pres[e][3]};
        const uint4 r = philox4x32_10_rk(make_uint4(cellid[e], sweep, (unsigned)K.chain, 0u), F.rk);
        const MoveAngles ga = move_angles(K.sigma, omc, uniform01(r.x), uniform01(r.y), uniform01(r.z));
        const float u3 = uniform01(r.w);
        Move v = move_length(a[e], K.me2h, K.me2l);
        move_direction_g(v, a[e], ga);
        const float floc = local_change_flat(v, a[e], nb[e], wv, pres[e], K.cdx, K.cdy, (flags & F_DMI) != 0,
                                             h[e].x, h[e].y, h[e].z);
        const float flong = longitudinal_change(v, K.p2, K.p4);
        const float fan = anisotropy_change(v, flags, K.k1, K.k2, K.ex, K.ey, K.ez);
        const float dl = floc + flong + fan - 4.f * log1p_move_s(v.tt, K.sigma);
        acc = dl + __logf(u3) < 0.f;
        if (acc) {
          const float4 mp = make_float4(v.mpx, v.mpy, v.mpz, a[e].w);
          tb[ql[e]] = mp;
          mblk[MMC_CK(A.ck, (long long)r0 * hx + ql[e], 0, S, kCkFusedState)] = mp;
        }
      }
      na += __popc(__ballot_sync(0xffffffffu, acc));
      nv += __popc(__ballot_sync(0xffffffffu, valid[e]));
    }
  }
  if (lane == 0) {
    wacc[w] = na;
    watt[w] = nv;
  }
  __syncthreads();                                     // the tile's rows are final; counts ready
  if (threadIdx.x == 0) {
    unsigned sa = 0, sv = 0;
#pragma unroll
    for (int w2 = 0; w2 < kFusedThreads / 32; ++w2) { sa += wacc[w2]; sv += watt[w2]; }
    if (sv) {
      atomicAdd(&F.st[c].win_acc, (unsigned long long)sa);
      atomicAdd(&F.st[c].win_att, (unsigned long long)sv);
    }
  }

  // 2. the forward row transforms of the four rows, M from the tiles
  const int p = w / 3, q = w - 3 * p;
  const int rA = 4 * tile + 2 * p, rB = rA + 1;
  const float Ms = (float)ch.Ms0d;
  const int ra = q == 1 ? rB : rA;
  const bool ha = ra < ny, hb = q == 2 && rB < ny;
  // cell x = 32 n1 + lane of row r: colour (lane + r) & 1, slot 16 n1 + lane / 2
  const float4 *ta = ((lane + ra) & 1) ? tb + (ra - r0) * hx : tr + (ra - r0 + 1) * hx;
  const float4 *tbb = ((lane + rB) & 1) ? tb + (rB - r0) * hx : tr + (rB - r0 + 1) * hx;
  float2 v[32];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) {
    const int sl = 16 * n1 + (lane >> 1);
    const bool in = 32 * n1 + lane < nx;
    float2 z = make_float2(0.f, 0.f);
    if (in && ha) {
      const float4 t = ta[sl];
      z = q == 2 ? make_float2(Ms * t.z, 0.f) : make_float2(Ms * t.x, Ms * t.y);
    }
    if (in && hb) z.y = Ms * tbb[sl].z;
    v[n1] = z;
  }
  __syncthreads();                                     // every warp holds its sequence: tiles -> warp buffers
  float2 *buf = sm + w * kW32Buf;
  dft32_lo16(v);
  w32_fwd_tail(v, buf, A.tw, lane);
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) buf[lane + 32 * k2] = v[k2];
  __syncwarp();
  float2 X[17], Y[17];
#pragma unroll
  for (int k2 = 0; k2 < 17; ++k2) {
    if (k2 == 16 && lane != 0) break;
    const int k = lane + 32 * k2;
    const float2 Z = v[k2], Zm = buf[(kW32N - k) & (kW32N - 1)];
    X[k2] = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
    Y[k2] = make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));
  }
  __syncthreads();
  const int cA = q == 2 ? 2 : 0, cB = q == 2 ? 2 : 1;
  const int oA = q == 1 ? 2 * p + 1 : 2 * p, oB = q == 0 ? 2 * p : 2 * p + 1;
#pragma unroll
  for (int k2 = 0; k2 < 17; ++k2) {
    if (k2 == 16 && lane != 0) break;
    const int k = lane + 32 * k2;
    sm[(cA * 4 + oA) * kW32TilePitch + k] = X[k2];
    sm[(cB * 4 + oB) * kW32TilePitch + k] = Y[k2];
  }
  __syncthreads();
  constexpr int per = kW32Half * 2;
  for (int i = threadIdx.x; i < 3 * per; i += blockDim.x) {
    const int comp = i / per, o = i - comp * per;
    const int kx = o >> 1, hh = o & 1;
    const float2 aa = sm[(comp * 4 + 2 * hh) * kW32TilePitch + kx];
    const float2 bb = sm[(comp * 4 + 2 * hh + 1) * kW32TilePitch + kx];
    *reinterpret_cast<float4 *>(A.S + w32_tile_pair(A, ch, comp, tile, o)) = make_float4(aa.x, aa.y, bb.x, bb.y);
  }
}

// The inverse row transforms of a tile of four rows fused with the red pass of
// the same rows: once a tile's field is in shared memory the red cells of its
// rows can move (their field is final, their black neighbours do not move in
// this pass).  After the transforms, one thread brings the tile's red rows and
// the black rows r0 - 1 .. r0 + 4 into the space the transposes used; the block
// writes h_eff of the black cells (for the fused black pass), then runs the red
// pass from shared memory with each red cell's field taken from the tile.
constexpr size_t kFieldTileBytes = 12 * 512 * sizeof(float);
constexpr size_t kFusedInvSmem = kFieldTileBytes + (size_t)10 * kFusedHx * sizeof(float4);
static_assert(kFusedInvSmem >= 6 * kW32Buf * sizeof(float2), "the buffers cover the warp buffers");
static_assert(kFieldTileBytes % 16 == 0, "bulk copy alignment");

__global__ void __launch_bounds__(kFusedThreads, 3) k_w32_rows_inv_red(FusedArgs F) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *sm = reinterpret_cast<float2 *>(smem_raw);
  float *ft = reinterpret_cast<float *>(smem_raw);                      // field tile [comp][row][x]
  float4 *tred = reinterpret_cast<float4 *>(smem_raw + kFieldTileBytes);  // red rows r0 .. r0 + nr - 1
  float4 *tblk = tred + 4 * kFusedHx;                                     // black rows r0 - 1 .. r0 + nr
  __shared__ uint64_t bar;
  __shared__ float4 skv[kChainKVec];
  __shared__ unsigned wacc[kFusedThreads / 32], watt[kFusedThreads / 32];
  const W32Args &A = F.W;
  const int c = w32_chain_of_block(A);
  const ChainDev &ch = A.chains[c];
  const int tile = (int)(blockIdx.x - A.blk_first[c]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = w / 3, q = w - 3 * p;
  const int nx = ch.nx, ny = ch.ny, hx = ch.hx;
  const int r0 = 4 * tile, nr = min(4, ny - r0);
  const long long S = (long long)ch.nrows * hx;
  if (threadIdx.x < kChainKVec) skv[threadIdx.x] = __ldg(reinterpret_cast<const float4 *>(A.chains + c) + threadIdx.x);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  {
    constexpr int per = kW32Half * 2;
    for (int i = threadIdx.x; i < 3 * per; i += blockDim.x) {
      const int comp = i / per, o = i - comp * per;
      const float4 t = *reinterpret_cast<const float4 *>(A.S + w32_tile_pair(A, ch, comp, tile, o));
      const int kx = o >> 1, r = 2 * (o & 1);
      sm[(comp * 4 + r) * kW32TilePitch + kx] = make_float2(t.x, t.y);
      sm[(comp * 4 + r + 1) * kW32TilePitch + kx] = make_float2(t.z, t.w);
    }
  }
  __syncthreads();
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
      const int km = kW32N - k;
      const float2 a = ta[km], b = tb[km];
      v[k2] = km == 512 ? make_float2(a.x, b.x) : make_float2(a.x + b.y, b.x - a.y);
    }
  }
  __syncthreads();
  w32_inv(v, sm + w * kW32Buf, A.tw, lane);
  __syncthreads();                                     // transposes done: the space is free
  if (threadIdx.x == 0) {
    fence_proxy_async_smem();
    const bool pby = (ch.pbc & 2) != 0;
    const int rb = r0 > 0 ? r0 - 1 : (pby ? ny - 1 : -1);
    const int ra = r0 + nr < ny ? r0 + nr : (pby ? 0 : -1);
    const unsigned row_b = (unsigned)hx * 16u;
    const float4 *mred = A.m + ch.m_off, *mblk = A.m + ch.m_off + S;
    mbar_arrive_expect_tx(&bar, 2u * (unsigned)nr * row_b + (rb >= 0 ? row_b : 0u) + (ra >= 0 ? row_b : 0u));
    const long long o0 = MMC_CKR(A.ck, (long long)r0 * hx, (long long)nr * hx, 0, S, kCkFusedCopy);
    bulk_g2s(tred, mred + o0, (unsigned)nr * row_b, &bar);
    bulk_g2s(tblk + hx, mblk + o0, (unsigned)nr * row_b, &bar);
    if (rb >= 0) bulk_g2s(tblk, mblk + MMC_CKR(A.ck, (long long)rb * hx, hx, 0, S, kCkFusedCopy), row_b, &bar);
    if (ra >= 0)
      bulk_g2s(tblk + (long long)(nr + 1) * hx, mblk + MMC_CKR(A.ck, (long long)ra * hx, hx, 0, S, kCkFusedCopy),
               row_b, &bar);
  }
  const float scale = 1.f / ((float)kW32N * (float)kW32N);
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) {
    const int x = lane + 32 * n2;
    ft[(cA * 4 + rA) * 512 + x] = v[n2].x * scale;
    ft[(cB * 4 + rB) * 512 + x] = v[n2].y * scale;
  }
  __syncthreads();
  const ChainK K = load_chain_vec(skv);
  const float mu0f = (float)mu0;
  // h_eff of the black cells, for the fused black pass
  const unsigned nslots = (unsigned)(nr * hx);
  for (unsigned qb = threadIdx.x; qb < nslots; qb += blockDim.x) {
    const int rl = (int)divq(qb, K.hx_m, K.hx_l), sl = (int)(qb - (unsigned)rl * (unsigned)hx);
    const int x = 2 * sl + ((r0 + rl + 1) & 1);
    if (x >= nx) continue;
    const float Hx = ft[(0 * 4 + rl) * 512 + x], Hy = ft[(1 * 4 + rl) * 512 + x], Hz = ft[(2 * 4 + rl) * 512 + x];
    A.heff[ch.h_off + S + MMC_CK(A.ck, (long long)r0 * hx + qb, 0, S, kCkDemagField)] = make_float4(
        ch.zee * (ch.Bx + mu0f * Hx), ch.zee * (ch.By + mu0f * Hy), ch.zee * (ch.Bz + mu0f * Hz), 0.f);
  }
  if (!mbar_wait(&bar, 0u, F.max_polls)) {
    if (threadIdx.x == 0) atomicExch(A.err, -3);      // MMC_ERR_TIMEOUT: the tile's red cells do not move
    const long long t0 = clock64();
    while (clock64() - t0 < (1LL << 21)) {
    }
    return;
  }
  // the red pass (colour 0) on the tile's cells
  const unsigned sweep = *F.sweep_base + F.sweep_off;
  const float omc = F.st[c].omc;
  const int pbc = K.pbc & 3, flags = K.flags;
  float4 *mredw = F.m + ch.m_off;
  unsigned na = 0, nv = 0;
#pragma unroll 1
  for (int e0 = 0; e0 < 6; e0 += 2) {
    bool valid[2];
    unsigned ql[2], cellid[2];
    float4 a[2], h[2], nb[2][4];
    float pres[2][4];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const unsigned qq = threadIdx.x + (unsigned)((e0 + e) * kFusedThreads);
      bool ok = qq < nslots;
      const int rl = ok ? (int)divq(qq, K.hx_m, K.hx_l) : 0;
      const int sl = (int)(qq - (unsigned)rl * (unsigned)hx);
      const int j = r0 + rl;
      const int pp = j & 1;
      const int i = 2 * sl + pp;
      ok = ok && (i < nx);
      valid[e] = ok;
      ql[e] = qq;
      cellid[e] = (unsigned)i + (unsigned)nx * (unsigned)j;
      if (ok) {
        a[e] = tred[qq];
        const float4 *O = tblk + (rl + 1) * hx + sl;
        const bool hl = i > 0 || (pbc & 1), hr = i < nx - 1 || (pbc & 1);
        const bool hu = j > 0 || (pbc & 2), hd = j < ny - 1 || (pbc & 2);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        nb[e][0] = hl ? O[i > 0 ? pp - 1 : hx - 1] : z4;
        nb[e][1] = hr ? O[i < nx - 1 ? pp : 1 - hx] : z4;
        nb[e][2] = hu ? O[-hx] : z4;
        nb[e][3] = hd ? O[hx] : z4;
        pres[e][0] = hl ? 1.f : 0.f;
        pres[e][1] = hr ? 1.f : 0.f;
        pres[e][2] = hu ? 1.f : 0.f;
        pres[e][3] = hd ? 1.f : 0.f;
        if (flags & F_GRAIN) {
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (nb[e][b].w != a[e].w) pres[e][b] *= K.gscale;
        }
        const float Hx = ft[(0 * 4 + rl) * 512 + i], Hy = ft[(1 * 4 + rl) * 512 + i], Hz = ft[(2 * 4 + rl) * 512 + i];
        h[e] = make_float4(ch.zee * (ch.Bx + mu0f * Hx), ch.zee * (ch.By + mu0f * Hy), ch.zee * (ch.Bz + mu0f * Hz), 0.f);
      }
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int acc = 0;
      if (valid[e]) {
        const float wv[4] = {K.wx * pres[e][0], K.wx * pres[e][1], K.wy * pres[e][2], K.wy * pres[e][3]};
        const uint4 r = philox4x32_10_rk(make_uint4(cellid[e], sweep, (unsigned)K.chain, 0u), F.rk);
        const MoveAngles ga = move_angles(K.sigma, omc, uniform01(r.x), uniform01(r.y), uniform01(r.z));
        const float u3 = uniform01(r.w);
        Move mv = move_length(a[e], K.me2h, K.me2l);
        move_direction_g(mv, a[e], ga);
        const float floc = local_change_flat(mv, a[e], nb[e], wv, pres[e], K.cdx, K.cdy, (flags & F_DMI) != 0,
                                             h[e].x, h[e].y, h[e].z);
        const float flong = longitudinal_change(mv, K.p2, K.p4);
        const float fan = anisotropy_change(mv, flags, K.k1, K.k2, K.ex, K.ey, K.ez);
        const float dl = floc + flong + fan - 4.f * log1p_move_s(mv.tt, K.sigma);
        acc = dl + __logf(u3) < 0.f;
        if (acc) mredw[MMC_CK(A.ck, (long long)r0 * hx + ql[e], 0, S, kCkFusedState)] = make_float4(mv.mpx, mv.mpy, mv.mpz, a[e].w);
      }
      na += __popc(__ballot_sync(0xffffffffu, acc));
      nv += __popc(__ballot_sync(0xffffffffu, valid[e]));
    }
  }
  if (lane == 0) {
    wacc[w] = na;
    watt[w] = nv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned sa = 0, sv = 0;
#pragma unroll
    for (int w2 = 0; w2 < kFusedThreads / 32; ++w2) { sa += wacc[w2]; sv += watt[w2]; }
    if (sv) {
      atomicAdd(&F.st[c].win_acc, (unsigned long long)sa);
      atomicAdd(&F.st[c].win_att, (unsigned long long)sv);
    }
  }
}

constexpr size_t kW32RowsSmem = 6 * kW32Buf * sizeof(float2);
constexpr size_t kW32ColsSmem = 3 * kW32Buf * sizeof(float2) + 4 * kW32TPitch * sizeof(float);
static_assert(kW32RowsSmem >= 12 * kW32TilePitch * sizeof(float2), "output tile fits the warp buffers");
static_assert((3 * kW32Buf * sizeof(float2)) % 16 == 0 && (kW32TPitch * 4) % 16 == 0, "bulk copy alignment");
static_assert(kW32RowsSmem >= 12 * kW32TilePitch * sizeof(float2), "input tile fits the warp buffers");
static_assert(kW32RowsSmem >= 12 * 512 * sizeof(float), "field tile fits the warp buffers");

static W32Args w32_args(const DemagLaunch &P) {
  W32Args A;
  A.chains = P.chains; A.m = P.m; A.tab = P.tab; A.ms = P.ms;
  A.S = reinterpret_cast<float2 *>(P.spec);
  A.nhatT = reinterpret_cast<const float *const *>(P.nhatT);
  A.tw = reinterpret_cast<const float2 *>(P.tw1024);
  A.heff = P.heff; A.Hd = P.Hd; A.Hd_chain = P.Hd_chain;
  A.err = P.err;
  A.ck = P.ck; A.nchains = P.nchains;
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  return A;
}

void launch_w32(const Launch &L, const DemagLaunch &P) {
  W32Args A = w32_args(P);
  if (P.ev) cudaEventRecord(P.ev[0], L.stream);
  k_w32_rows_fwd<<<P.rows_blocks, 192, kW32RowsSmem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[1], L.stream);
  A.blk_chain = P.cols_chain; A.blk_first = P.cols_first;
  k_w32_cols<<<P.cols_blocks, 96, kW32ColsSmem, L.stream>>>(A, *static_cast<const CUtensorMap *>(P.tmap_spec));
  if (P.ev) cudaEventRecord(P.ev[2], L.stream);
  A.blk_chain = P.rows_chain; A.blk_first = P.rows_first;
  k_w32_rows_inv<<<P.rows_blocks, 192, kW32RowsSmem, L.stream>>>(A);
  if (P.ev) cudaEventRecord(P.ev[3], L.stream);
  *L.counter += 3;
}

void launch_w32_stage(const Launch &L, const DemagLaunch &P, int stage) {
  W32Args A = w32_args(P);
  if (stage == 0) {
    k_w32_rows_fwd<<<P.rows_blocks, 192, kW32RowsSmem, L.stream>>>(A);
  } else if (stage == 1) {
    A.blk_chain = P.cols_chain; A.blk_first = P.cols_first;
    k_w32_cols<<<P.cols_blocks, 96, kW32ColsSmem, L.stream>>>(A, *static_cast<const CUtensorMap *>(P.tmap_spec));
  } else {
    k_w32_rows_inv<<<P.rows_blocks, 192, kW32RowsSmem, L.stream>>>(A);
  }
  ++*L.counter;
}

static FusedArgs fused_args(const DemagLaunch &P, const SweepLaunch &Q) {
  FusedArgs F;
  F.W = w32_args(P);
  F.m = Q.m;
  F.st = Q.st;
  F.heff = Q.heff;
  F.sweep_base = Q.sweep_base;
  F.sweep_off = Q.sweep_off;
  unsigned k0 = Q.key0, k1 = Q.key1;
  for (int r = 0; r < 10; ++r) {
    F.rk[2 * r] = k0;
    F.rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  F.max_polls = Q.max_polls;
  return F;
}

void launch_w32_rows_inv_red(const Launch &L, const DemagLaunch &P, const SweepLaunch &Q) {
  FusedArgs F = fused_args(P, Q);
  k_w32_rows_inv_red<<<P.rows_blocks, kFusedThreads, kFusedInvSmem, L.stream>>>(F);
  ++*L.counter;
}

void launch_w32_black_rows_fwd(const Launch &L, const DemagLaunch &P, const SweepLaunch &Q) {
  FusedArgs F;
  F.W = w32_args(P);
  F.m = Q.m;
  F.st = Q.st;
  F.heff = Q.heff;
  F.sweep_base = Q.sweep_base;
  F.sweep_off = Q.sweep_off;
  unsigned k0 = Q.key0, k1 = Q.key1;
  for (int r = 0; r < 10; ++r) {
    F.rk[2 * r] = k0;
    F.rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  F.max_polls = Q.max_polls;
  k_w32_black_rows_fwd<<<P.rows_blocks, kFusedThreads, kFusedSmem, L.stream>>>(F);
  ++*L.counter;
}

cudaError_t w32_set_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_w32_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kW32RowsSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_w32_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kW32RowsSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_w32_black_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_w32_rows_inv_red, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedInvSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_w32_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kW32ColsSmem);
}

}  // namespace mmc
