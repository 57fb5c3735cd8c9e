// Sublattice pass of the MMC iteration (Sec. II) on all chains of a batch.
//
// Data layout (per chain): m is stored split by checkerboard colour.  Colour c
// of row r = j + ny*k holds the cells i = 2 s + ((j + k + c) & 1), s in
// [0, hx), hx = (nx + 1) / 2, as float4 (mx, my, mz, grain id) at
// m_off + c * nrows * hx + r * hx + s.  The neighbours of a colour-c cell are all
// in the other colour's array: the in-row ones at slots s - 1 + p and s + p
// (p = (j + k + c) & 1), the ones in rows j +- 1 and planes k +- 1 at slot s.
// A block covers 256 consecutive slots of one chain (128 threads, two cells
// each), so a launch covers every chain of the batch.
//
// Per cell: Philox4x32-10 at counter (cell, sweep, chain, 0) gives u0..u3;
// the move is a rotation uniform on the cap of half-angle theta about m/|m|
// (cos = 1 - u0 (1 - cos theta), phi = 2 pi u1, basis of Duff et al. 2017)
// times a length factor 1 + sigma (2 u2 - 1); the energy change in units of kT
// is exchange + DMI (pair sums, Eqs. 10, 15) + anisotropy (Eq. 11 / 12) +
// Zeeman and frozen demag field (Eq. 14) + longitudinal (Eq. 7); the move is
// accepted iff dF/kT - 4 ln(m'/m) + ln u3 < 0 (Eq. 5).
#include <algorithm>
#include <cstdio>

#include "mmc_internal.h"
#include "philox.cuh"
#include "tma.cuh"
#include "trial.cuh"

namespace mmc {

struct SweepArgs {
  const ChainDev *chains;
  ChainState *st;
  const int2 *blk_desc;     // per block: (chain, block index within the chain)
  int blk_base;
  float4 *m;
  const float4 *heff;
  const float4 *tab;        // per-cell tables, 3 float4 arrays per chain (split layout)
  const unsigned *sweep_base;
  unsigned sweep_off;
  unsigned key0, key1;
  int color;
  float omc_override;       // >= 0: use this 1 - cos(theta) (diagnostic pass)
  float *dec_dbg;
  signed char *acc_dbg;
  int nstripes, stripe;     // nstripes > 1: the band of rows [r0, r1) of the stripe only
  unsigned rk[20];          // Philox round keys of (key0, key1), see philox4x32_10_rk
  // banded pass (k_sweep_band): work items [i0, i1) of the item table
  const int4 *items;        // per band: (chain, first row, rows, 0)
  int i0, i1;
  int stage_own, stage_other;   // float4 capacity of a stage's own-colour and other-colour tiles
  unsigned max_polls;       // bound of a wait for a band's copies
  int *err;                 // device error word (MMC_ERR_TIMEOUT on a wait that gave up)
  int wait_test;            // test hook: every band's barrier waits for 16 bytes no copy delivers
  // checked builds (checked.cuh): the record and the table sizes indices are checked against
  MmcCheck *ck;
  int blk_total, nchains, nitems;
};

// A thread handles kSweepCells cells of its block's 256 slots (slot t + j 128):
// the loads of all of them are issued before any is computed, so each thread
// keeps two independent trials in flight and the block prologue (block table,
// chain constants) is paid once per two cells.
constexpr int kSweepCells = 2;
constexpr int kSweepThreads = kSweepBlock / kSweepCells;

// FLAT: every chain of the launch is one cell thick (nz = 1), so the z
// neighbours, their loads and registers drop out at compile time.  Seven
// blocks per SM for uniform chains (72 registers): the pass waits on its cell
// and neighbour loads, and the extra warps hide that latency better than six
// blocks (80 registers) or eight (64 registers, more spills) did on GB300.
template <bool PERCELL, bool DEBUG, bool FLAT>
__global__ void __launch_bounds__(kSweepThreads, PERCELL ? 5 : 7) k_sweep_pass(SweepArgs A) {
  pdl_enter();
  const int2 bd = A.blk_desc[MMC_CK(A.ck, A.blk_base + (int)blockIdx.x, 0, A.blk_total, kCkSweepBlock)];
  const int c = (int)MMC_CK(A.ck, bd.x, 0, A.nchains, kCkSweepBlock);
  const ChainK K = load_chain(A.chains + c);
  const int nx = K.nx, ny = K.ny, nz = FLAT ? 1 : K.nz, hx = K.hx;
  const int pbc = FLAT ? (K.pbc & 3) : K.pbc;
  // a chain has fewer than 2^31 cells: 32-bit slot arithmetic
  const unsigned S32 = (unsigned)K.nrows * (unsigned)hx;
  const long long S = (long long)S32;
  const unsigned q0 = (unsigned)bd.y * (unsigned)kSweepBlock + threadIdx.x;
  const int color = A.color;
  const int flags = K.flags;
  float4 *mc = A.m + K.m_off + (long long)color * S;
  const float4 *mo = A.m + K.m_off + (long long)(1 - color) * S;
  const float omc = A.omc_override >= 0.f ? A.omc_override : A.st[c].omc;
  const unsigned sweep = *A.sweep_base + A.sweep_off;
  // the slots of the pass: all, or the rows [r0, r1) of one band (the demag
  // field is then recomputed between bands); a block outside the band leaves
  // before any barrier
  unsigned lo = 0, hi = S32;
  if (A.nstripes > 1) {
    const unsigned long long nr = (unsigned long long)K.nrows;
    lo = (unsigned)((unsigned long long)A.stripe * nr / (unsigned)A.nstripes) * (unsigned)hx;
    hi = (unsigned)((unsigned long long)(A.stripe + 1) * nr / (unsigned)A.nstripes) * (unsigned)hx;
    const unsigned b0 = (unsigned)bd.y * (unsigned)kSweepBlock;
    if (b0 >= hi || b0 + (unsigned)kSweepBlock <= lo) return;
  }

  // 1. indices and loads of every cell of this thread
  bool valid[kSweepCells];
  unsigned qq[kSweepCells], cellid[kSweepCells];
  float4 a[kSweepCells], h[kSweepCells];
  float4 nb[kSweepCells][6];
  float w[kSweepCells][6];
  CellMat M[kSweepCells];
#pragma unroll
  for (int e = 0; e < kSweepCells; ++e) {
    const unsigned q32 = q0 + (unsigned)(e * kSweepThreads);
    bool ok = q32 >= lo && q32 < hi;
    const int row = ok ? (int)divq(q32, K.hx_m, K.hx_l) : 0;
    const int s = (int)(q32 - (unsigned)row * (unsigned)hx);
    const int k = FLAT ? 0 : (int)divq((unsigned)row, K.ny_m, K.ny_l), j = row - k * ny;
    const int p = (j + k + color) & 1;
    const int i = 2 * s + p;
    ok = ok && (i < nx);
    valid[e] = ok;
    qq[e] = q32;
    cellid[e] = (unsigned)i + (unsigned)nx * (unsigned)row;
    if (ok) {
      a[e] = mc[MMC_CK(A.ck, q32, 0, S, kCkSweepCell)];
      load_neighbours(pbc, (flags & F_GRAIN) != 0, K.gscale, nx, ny, nz, hx, mo, a[e], i, j, k, row, s, p, nb[e], w[e],
                      A.ck, S);
      M[e] = cell_material<PERCELL>(K, A.tab, S, (long long)color * S + q32, A.ck);
      if (flags & F_DEMAG) h[e] = A.heff[K.h_off + (long long)color * S + MMC_CK(A.ck, q32, 0, S, kCkSweepField)];
      else h[e] = make_float4(M[e].zee * K.Bx, M[e].zee * K.By, M[e].zee * K.Bz, 0.f);
    }
  }

  // 2. the trials
  int accepted[kSweepCells];
#pragma unroll
  for (int e = 0; e < kSweepCells; ++e) {
    accepted[e] = 0;
    if (!valid[e]) continue;
    const float wx = K.wx * M[e].bs, wy = K.wy * M[e].bs, wz = K.wz * M[e].bs;
    const float cdx = K.cdx * M[e].bs, cdy = K.cdy * M[e].bs;
    const uint4 r = philox4x32_10(make_uint4(cellid[e], sweep, (unsigned)K.chain, 0u), make_uint2(A.key0, A.key1));
    const float u0 = uniform01(r.x), u1 = uniform01(r.y), u2 = uniform01(r.z), u3 = uniform01(r.w);
    Move v = move_length(a[e], M[e].me2h, M[e].me2l);
    move_direction(v, a[e], M[e].sigma, omc, u0, u1, u2);
    const float fex = exchange_change(v, a[e], nb[e], w[e], wx, wy, wz, !FLAT && nz > 1);
    const float flin = linear_change(v, nb[e], w[e], cdx, cdy, (flags & F_DMI) != 0, h[e].x, h[e].y, h[e].z);
    const float flong = longitudinal_change(v, M[e].p2, M[e].p4);
    const float fan = anisotropy_change(v, flags, M[e].k1, M[e].k2, M[e].ex, M[e].ey, M[e].ez);
    const float dF = fex + flin + flong + fan;
    const float lg = log1p_move(v.tt);
    const float dl = dF - 4.f * lg;
    // ln u3 < 0: a non-positive dl accepts whatever u3 is, so its log is skipped
    float dec;
    if (DEBUG || dl > 0.f) dec = dl + __logf(u3);
    else dec = dl;
    accepted[e] = dec < 0.f;
    if (accepted[e]) mc[MMC_CK(A.ck, qq[e], 0, S, kCkSweepCell)] = make_float4(v.mpx, v.mpy, v.mpz, a[e].w);
    if (DEBUG) {
      const long long cd = MMC_CK(A.ck, cellid[e], 0, (long long)K.nrows * nx, kCkSweepDebug);
      A.dec_dbg[cd] = dec;
      A.acc_dbg[cd] = (signed char)accepted[e];
    }
  }

  // acceptance counts: warp ballots, then one atomic per block
  __shared__ unsigned wacc[kSweepThreads / 32], watt[kSweepThreads / 32];
  unsigned na = 0, nv = 0;
#pragma unroll
  for (int e = 0; e < kSweepCells; ++e) {
    na += __popc(__ballot_sync(0xffffffffu, accepted[e]));
    nv += __popc(__ballot_sync(0xffffffffu, valid[e]));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    wacc[warp] = na;
    watt[warp] = nv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned sa = 0, sv = 0;
#pragma unroll
    for (int w2 = 0; w2 < kSweepThreads / 32; ++w2) { sa += wacc[w2]; sv += watt[w2]; }
    if (sv) {
      atomicAdd(&A.st[c].win_acc, (unsigned long long)sa);
      atomicAdd(&A.st[c].win_att, (unsigned long long)sv);
    }
  }
}

// One-cell-thick chains (every chain of the launch has nz = 1): the same pass
// with the work per cell cut down.  The chain constants are read once per block
// into shared memory; the Philox round keys come precomputed in the kernel
// parameters; the four in-plane neighbours are found by offsets from the cell's
// slot in the other colour (s - 1 + p, s + p in the row, s in the rows j -+ 1,
// with the periodic wrap at the edges); exchange, DMI and the field act through
// one local vector (local_change_flat).
template <bool PERCELL, bool DEBUG, int MINB>
__global__ void __launch_bounds__(kSweepThreads, MINB) k_sweep_flat(SweepArgs A) {
  pdl_enter();
  __shared__ float4 skv[kChainKVec];
  __shared__ unsigned wacc[kSweepThreads / 32], watt[kSweepThreads / 32];
  const int2 bd = A.blk_desc[MMC_CK(A.ck, A.blk_base + (int)blockIdx.x, 0, A.blk_total, kCkSweepBlock)];
  const int c = (int)MMC_CK(A.ck, bd.x, 0, A.nchains, kCkSweepBlock);
  if (threadIdx.x < kChainKVec) skv[threadIdx.x] = __ldg(reinterpret_cast<const float4 *>(A.chains + c) + threadIdx.x);
  __syncthreads();
  const ChainK K = load_chain_vec(skv);
  const int nx = K.nx, ny = K.ny, hx = K.hx;
  const int pbc = K.pbc & 3;
  const unsigned S32 = (unsigned)K.nrows * (unsigned)hx;
  const long long S = (long long)S32;
  const unsigned q0 = (unsigned)bd.y * (unsigned)kSweepBlock + threadIdx.x;
  const int color = A.color;
  const int flags = K.flags;
  float4 *mc = A.m + K.m_off + (long long)color * S;
  const float4 *mo = A.m + K.m_off + (long long)(1 - color) * S;
  const float omc = A.omc_override >= 0.f ? A.omc_override : A.st[c].omc;
  const unsigned sweep = *A.sweep_base + A.sweep_off;
  unsigned lo = 0, hi = S32;
  if (A.nstripes > 1) {
    const unsigned long long nr = (unsigned long long)K.nrows;
    lo = (unsigned)((unsigned long long)A.stripe * nr / (unsigned)A.nstripes) * (unsigned)hx;
    hi = (unsigned)((unsigned long long)(A.stripe + 1) * nr / (unsigned)A.nstripes) * (unsigned)hx;
    const unsigned b0 = (unsigned)bd.y * (unsigned)kSweepBlock;
    if (b0 >= hi || b0 + (unsigned)kSweepBlock <= lo) return;     // the whole block, before the next barrier
  }
  const bool grain = (flags & F_GRAIN) != 0;

  // 1. indices and loads of every cell of this thread
  bool valid[kSweepCells];
  unsigned qq[kSweepCells], cellid[kSweepCells];
  float4 a[kSweepCells], h[kSweepCells];
  float4 nb[kSweepCells][4];
  float pres[kSweepCells][4];
  CellMat M[kSweepCells];
#pragma unroll
  for (int e = 0; e < kSweepCells; ++e) {
    const unsigned q32 = q0 + (unsigned)(e * kSweepThreads);
    bool ok = q32 >= lo && q32 < hi;
    const int j = ok ? (int)divq(q32, K.hx_m, K.hx_l) : 0;     // row (one cell thick: j)
    const int s = (int)(q32 - (unsigned)j * (unsigned)hx);
    const int p = (j + color) & 1;
    const int i = 2 * s + p;
    ok = ok && (i < nx);
    valid[e] = ok;
    qq[e] = q32;
    cellid[e] = (unsigned)i + (unsigned)nx * (unsigned)j;
    if (ok) {
      a[e] = mc[MMC_CK(A.ck, q32, 0, S, kCkSweepCell)];
      // the other colour's slots of the -x, +x, -y, +y neighbours, relative to
      // slot s of row j (periodic axes have even extents)
      const long long pb = (long long)j * hx + s;
      const float4 *P = mo + pb;
      const bool hl = i > 0 || (pbc & 1), hr = i < nx - 1 || (pbc & 1);
      const bool hu = j > 0 || (pbc & 2), hd = j < ny - 1 || (pbc & 2);
      const int ol = i > 0 ? p - 1 : hx - 1;
      const int orr = i < nx - 1 ? p : 1 - hx;
      const int ou = j > 0 ? -hx : (ny - 1) * hx;
      const int od = j < ny - 1 ? hx : -(ny - 1) * hx;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      nb[e][0] = hl ? P[MMC_CK(A.ck, ol, -pb, S - pb, kCkSweepNeighbour)] : z4;
      nb[e][1] = hr ? P[MMC_CK(A.ck, orr, -pb, S - pb, kCkSweepNeighbour)] : z4;
      nb[e][2] = hu ? P[MMC_CK(A.ck, ou, -pb, S - pb, kCkSweepNeighbour)] : z4;
      nb[e][3] = hd ? P[MMC_CK(A.ck, od, -pb, S - pb, kCkSweepNeighbour)] : z4;
      pres[e][0] = hl ? 1.f : 0.f;
      pres[e][1] = hr ? 1.f : 0.f;
      pres[e][2] = hu ? 1.f : 0.f;
      pres[e][3] = hd ? 1.f : 0.f;
      if (grain) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (nb[e][b].w != a[e].w) pres[e][b] *= K.gscale;
      }
      M[e] = cell_material<PERCELL>(K, A.tab, S, (long long)color * S + q32, A.ck);
      if (flags & F_DEMAG) h[e] = A.heff[K.h_off + (long long)color * S + MMC_CK(A.ck, q32, 0, S, kCkSweepField)];
      else h[e] = make_float4(M[e].zee * K.Bx, M[e].zee * K.By, M[e].zee * K.Bz, 0.f);
    }
  }

  // 2. the random numbers and the parts of the moves that do not depend on m,
  // while the loads are in flight
  MoveAngles ga[kSweepCells];
  float u3v[kSweepCells], lgv[kSweepCells];
#pragma unroll
  for (int e = 0; e < kSweepCells; ++e) {
    const uint4 r = philox4x32_10_rk(make_uint4(cellid[e], sweep, (unsigned)K.chain, 0u), A.rk);
    const float sig = PERCELL ? (valid[e] ? M[e].sigma : 0.f) : K.sigma;
    ga[e] = move_angles(sig, omc, uniform01(r.x), uniform01(r.y), uniform01(r.z));
    u3v[e] = uniform01(r.w);
    lgv[e] = PERCELL ? log1p_move(ga[e].tt) : log1p_move_s(ga[e].tt, K.sigma);
  }

  // 3. the trials
  int accepted[kSweepCells];
#pragma unroll
  for (int e = 0; e < kSweepCells; ++e) {
    accepted[e] = 0;
    if (!valid[e]) continue;
    const float wx = K.wx * M[e].bs, wy = K.wy * M[e].bs;
    const float w[4] = {wx * pres[e][0], wx * pres[e][1], wy * pres[e][2], wy * pres[e][3]};
    const float u3 = u3v[e];
    Move v = move_length(a[e], M[e].me2h, M[e].me2l);
    move_direction_g(v, a[e], ga[e]);
    const float floc = local_change_flat(v, a[e], nb[e], w, pres[e], K.cdx * M[e].bs, K.cdy * M[e].bs,
                                         (flags & F_DMI) != 0, h[e].x, h[e].y, h[e].z);
    const float flong = longitudinal_change(v, M[e].p2, M[e].p4);
    const float fan = anisotropy_change(v, flags, M[e].k1, M[e].k2, M[e].ex, M[e].ey, M[e].ez);
    const float dF = floc + flong + fan;
    const float dl = dF - 4.f * lgv[e];
    // ln u3 < 0: accept iff dl + ln u3 < 0 (taken for every cell: no divergent branch)
    const float dec = dl + __logf(u3);
    accepted[e] = dec < 0.f;
    if (accepted[e]) mc[MMC_CK(A.ck, qq[e], 0, S, kCkSweepCell)] = make_float4(v.mpx, v.mpy, v.mpz, a[e].w);
    if (DEBUG) {
      const long long cd = MMC_CK(A.ck, cellid[e], 0, (long long)nx * K.nrows, kCkSweepDebug);
      A.dec_dbg[cd] = dec;
      A.acc_dbg[cd] = (signed char)accepted[e];
    }
  }

  unsigned na = 0, nv = 0;
#pragma unroll
  for (int e = 0; e < kSweepCells; ++e) {
    na += __popc(__ballot_sync(0xffffffffu, accepted[e]));
    nv += __popc(__ballot_sync(0xffffffffu, valid[e]));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    wacc[warp] = na;
    watt[warp] = nv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned sa = 0, sv = 0;
#pragma unroll
    for (int w2 = 0; w2 < kSweepThreads / 32; ++w2) { sa += wacc[w2]; sv += watt[w2]; }
    if (sv) {
      atomicAdd(&A.st[c].win_acc, (unsigned long long)sa);
      atomicAdd(&A.st[c].win_att, (unsigned long long)sv);
    }
  }
}

// Banded pass with shared-memory halo tiles, for batches of uniform one-cell-
// thick chains.  Work items are bands of R rows of one chain (R hx <= 512 slots);
// a block walks the items blockIdx.x, blockIdx.x + gridDim.x, ... and, while it
// computes one band, one thread has the bulk-copy engine bring the next band
// into the other of two shared-memory stages: the band's own-colour rows, the
// other colour's rows r0 - 1 .. r0 + R (the halo rows, wrapped on periodic y
// axes, left out at open edges) and the h_eff rows.  Every neighbour of a band's
// cell is then in shared memory: the -x, +x neighbours in the other colour's
// row at slots s - 1 + p, s + p, the -y, +y neighbours in the rows above and
// below at slot s.  The moves are those of k_sweep_flat, cell for cell.
constexpr int kBandThreads = 256;
constexpr int kBandCells = 2;                // cells per thread: 512 slots per band at most

struct BandStage {
  float4 *own, *other, *heff;
};

__device__ __forceinline__ BandStage band_stage(unsigned char *base, int k, const SweepArgs &A) {
  float4 *b = reinterpret_cast<float4 *>(base) + (size_t)k * (2 * A.stage_own + A.stage_other);
  return BandStage{b, b + A.stage_own, b + A.stage_own + A.stage_other};
}

// one thread: arm bar with the bytes of item `it` and start its copies into stage g
// (extra: bytes the barrier waits for beyond the copies, a test hook whose
// barrier never completes)
__device__ __forceinline__ void band_issue(const SweepArgs &A, int4 it, const BandStage &g, uint64_t *bar,
                                           unsigned extra) {
  const ChainDev &ch = A.chains[it.x];
  const bool demag = (ch.flags & F_DEMAG) != 0;
  const int hx = ch.hx, ny = ch.ny, r0 = it.y, nr = it.z;
  const long long S = (long long)ch.nrows * hx;
  const float4 *own = A.m + ch.m_off + (long long)A.color * S;
  const float4 *oth = A.m + ch.m_off + (long long)(1 - A.color) * S;
  const unsigned row_b = (unsigned)hx * 16u;
  const bool pby = (ch.pbc & 2) != 0;
  const int rb = r0 > 0 ? r0 - 1 : (pby ? ny - 1 : -1);
  const int ra = r0 + nr < ny ? r0 + nr : (pby ? 0 : -1);
  unsigned bytes = 2u * (unsigned)nr * row_b + (rb >= 0 ? row_b : 0u) + (ra >= 0 ? row_b : 0u);
  if (demag) bytes += (unsigned)nr * row_b;
  mbar_arrive_expect_tx(bar, bytes + extra);
  const long long band = MMC_CKR(A.ck, (long long)r0 * hx, (long long)nr * hx, 0, S, kCkBandCopy);
  bulk_g2s(g.own, own + band, (unsigned)nr * row_b, bar);
  bulk_g2s(g.other + hx, oth + band, (unsigned)nr * row_b, bar);
  if (rb >= 0) bulk_g2s(g.other, oth + MMC_CKR(A.ck, (long long)rb * hx, hx, 0, S, kCkBandCopy), row_b, bar);
  if (ra >= 0)
    bulk_g2s(g.other + (long long)(nr + 1) * hx, oth + MMC_CKR(A.ck, (long long)ra * hx, hx, 0, S, kCkBandCopy), row_b,
             bar);
  if (demag) bulk_g2s(g.heff, A.heff + ch.h_off + (long long)A.color * S + band, (unsigned)nr * row_b, bar);
}

template <bool DEBUG>
__global__ void __launch_bounds__(kBandThreads, 3) k_sweep_band(SweepArgs A) {
  extern __shared__ __align__(16) unsigned char band_smem[];
  __shared__ uint64_t bar[2];
  __shared__ float4 skv[kChainKVec];
  __shared__ unsigned wacc[2][kBandThreads / 32], watt[2][kBandThreads / 32];
  __shared__ int abort_band;
  const int G = (int)gridDim.x;
  const unsigned extra = A.wait_test ? 16u : 0u;
  const unsigned sweep = *A.sweep_base + A.sweep_off;
  const int color = A.color;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    abort_band = 0;
  }
  __syncthreads();
  int item = A.i0 + (int)blockIdx.x;
  if (threadIdx.x == 0 && item < A.i1)
    band_issue(A, A.items[MMC_CK(A.ck, item, 0, A.nitems, kCkBandItem)], band_stage(band_smem, 0, A), &bar[0], extra);
  int prev_c = -1, k = 0;
  for (; item < A.i1; ++k, item += G) {
    const int st = k & 1;
    const int4 it = A.items[MMC_CK(A.ck, item, 0, A.nitems, kCkBandItem)];
    if (threadIdx.x == 0) {
      const int nxt = item + G;
      if (nxt < A.i1) {
        fence_proxy_async_smem();
        band_issue(A, A.items[MMC_CK(A.ck, nxt, 0, A.nitems, kCkBandItem)], band_stage(band_smem, st ^ 1, A),
                   &bar[st ^ 1], extra);
      }
      if (prev_c >= 0) {                      // counts of the previous band
        unsigned sa = 0, sv = 0;
#pragma unroll
        for (int w2 = 0; w2 < kBandThreads / 32; ++w2) { sa += wacc[st ^ 1][w2]; sv += watt[st ^ 1][w2]; }
        if (sv) {
          atomicAdd(&A.st[prev_c].win_acc, (unsigned long long)sa);
          atomicAdd(&A.st[prev_c].win_att, (unsigned long long)sv);
        }
      }
    }
    if (threadIdx.x < kChainKVec) skv[threadIdx.x] = __ldg(reinterpret_cast<const float4 *>(A.chains + it.x) + threadIdx.x);
    if (!mbar_wait(&bar[st], (unsigned)(k >> 1) & 1u, A.max_polls)) {
      abort_band = 1;
      atomicExch(A.err, (int)MMC_ERR_TIMEOUT_CODE);
    }
    __syncthreads();
    if (abort_band) break;
    const ChainK K = load_chain_vec(skv);
    const int c = it.x, r0 = it.y, nr = it.z;
    const int nx = K.nx, ny = K.ny, hx = K.hx;
    const int pbc = K.pbc & 3;
    const long long S = (long long)K.nrows * hx;
    float4 *mc = A.m + K.m_off + (long long)color * S;
    const BandStage g = band_stage(band_smem, st, A);
    const float omc = A.omc_override >= 0.f ? A.omc_override : A.st[c].omc;
    const int flags = K.flags;
    const unsigned nslots = (unsigned)(nr * hx);

    bool valid[kBandCells];
    unsigned ql[kBandCells], cellid[kBandCells];
    float4 a[kBandCells], h[kBandCells], nb[kBandCells][4];
    float pres[kBandCells][4];
#pragma unroll
    for (int e = 0; e < kBandCells; ++e) {
      const unsigned q = threadIdx.x + (unsigned)(e * kBandThreads);
      bool ok = q < nslots;
      const int rl = ok ? (int)divq(q, K.hx_m, K.hx_l) : 0;
      const int s = (int)(q - (unsigned)rl * (unsigned)hx);
      const int j = r0 + rl;
      const int p = (j + color) & 1;
      const int i = 2 * s + p;
      ok = ok && (i < nx);
      valid[e] = ok;
      ql[e] = q;
      cellid[e] = (unsigned)i + (unsigned)nx * (unsigned)j;
      if (ok) {
        a[e] = g.own[q];
        const float4 *O = g.other + (rl + 1) * hx + s;
        const bool hl = i > 0 || (pbc & 1), hr = i < nx - 1 || (pbc & 1);
        const bool hu = j > 0 || (pbc & 2), hd = j < ny - 1 || (pbc & 2);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        nb[e][0] = hl ? O[i > 0 ? p - 1 : hx - 1] : z4;
        nb[e][1] = hr ? O[i < nx - 1 ? p : 1 - hx] : z4;
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
        h[e] = (flags & F_DEMAG) ? g.heff[q] : make_float4(K.zee * K.Bx, K.zee * K.By, K.zee * K.Bz, 0.f);
      }
    }
    int accepted[kBandCells];
#pragma unroll
    for (int e = 0; e < kBandCells; ++e) {
      accepted[e] = 0;
      if (!valid[e]) continue;
      const float w[4] = {K.wx * pres[e][0], K.wx * pres[e][1], K.wy * pres[e][2], K.wy * pres[e][3]};
      const uint4 r = philox4x32_10_rk(make_uint4(cellid[e], sweep, (unsigned)K.chain, 0u), A.rk);
      const MoveAngles ga = move_angles(K.sigma, omc, uniform01(r.x), uniform01(r.y), uniform01(r.z));
      const float u3 = uniform01(r.w);
      Move v = move_length(a[e], K.me2h, K.me2l);
      move_direction_g(v, a[e], ga);
      const float floc = local_change_flat(v, a[e], nb[e], w, pres[e], K.cdx, K.cdy, (flags & F_DMI) != 0,
                                           h[e].x, h[e].y, h[e].z);
      const float flong = longitudinal_change(v, K.p2, K.p4);
      const float fan = anisotropy_change(v, flags, K.k1, K.k2, K.ex, K.ey, K.ez);
      const float dl = floc + flong + fan - 4.f * log1p_move_s(v.tt, K.sigma);
      const float dec = dl + __logf(u3);
      accepted[e] = dec < 0.f;
      const unsigned qg = (unsigned)r0 * (unsigned)hx + ql[e];
      if (accepted[e]) mc[MMC_CK(A.ck, qg, 0, S, kCkSweepCell)] = make_float4(v.mpx, v.mpy, v.mpz, a[e].w);
      if (DEBUG) {
        const long long cd = MMC_CK(A.ck, cellid[e], 0, (long long)nx * K.nrows, kCkSweepDebug);
        A.dec_dbg[cd] = dec;
        A.acc_dbg[cd] = (signed char)accepted[e];
      }
    }
    unsigned na = 0, nv = 0;
#pragma unroll
    for (int e = 0; e < kBandCells; ++e) {
      na += __popc(__ballot_sync(0xffffffffu, accepted[e]));
      nv += __popc(__ballot_sync(0xffffffffu, valid[e]));
    }
    if ((threadIdx.x & 31) == 0) {
      wacc[st][threadIdx.x >> 5] = na;
      watt[st][threadIdx.x >> 5] = nv;
    }
    prev_c = c;
    __syncthreads();                          // stage st, skv and the counts are read
  }
  if (abort_band) {
    // copies of this band and of the next may still be in flight into the
    // block's shared memory: give them a fixed time (about a millisecond, far
    // beyond a copy's latency) to land before the block exits
    const long long t0 = clock64();
    while (clock64() - t0 < (1LL << 21)) {
    }
    return;
  }
  if (threadIdx.x == 0 && prev_c >= 0) {
    const int st = (k - 1) & 1;
    unsigned sa = 0, sv = 0;
#pragma unroll
    for (int w2 = 0; w2 < kBandThreads / 32; ++w2) { sa += wacc[st][w2]; sv += watt[st][w2]; }
    if (sv) {
      atomicAdd(&A.st[prev_c].win_acc, (unsigned long long)sa);
      atomicAdd(&A.st[prev_c].win_att, (unsigned long long)sv);
    }
  }
}

size_t band_smem_bytes(int stage_own, int stage_other) {
  return (size_t)2 * (2 * stage_own + stage_other) * sizeof(float4);
}

cudaError_t band_set_smem(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_sweep_band<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_sweep_band<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int band_blocks_per_sm(size_t bytes) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_band<false>, kBandThreads, bytes) != cudaSuccess)
    return 1;
  return n < 1 ? 1 : n;
}

void launch_sweep_pass(const Launch &L, const SweepLaunch &P) {
  SweepArgs A;
  A.chains = P.chains; A.st = P.st; A.blk_desc = P.blk_desc;
  A.blk_base = P.blk_base;
  A.m = P.m; A.heff = P.heff; A.tab = P.tab; A.sweep_base = P.sweep_base;
  A.sweep_off = P.sweep_off; A.key0 = P.key0; A.key1 = P.key1; A.color = P.color;
  A.omc_override = P.omc_override; A.dec_dbg = P.dec_dbg; A.acc_dbg = P.acc_dbg;
  A.nstripes = P.nstripes; A.stripe = P.stripe;
  {
    unsigned k0 = P.key0, k1 = P.key1;
    for (int r = 0; r < 10; ++r) {
      A.rk[2 * r] = k0;
      A.rk[2 * r + 1] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
  A.items = P.items; A.i0 = P.i0; A.i1 = P.i1;
  A.stage_own = P.stage_own; A.stage_other = P.stage_other;
  A.max_polls = P.max_polls; A.err = P.err; A.wait_test = P.wait_test;
  A.ck = P.ck; A.blk_total = P.blk_total; A.nchains = P.nchains; A.nitems = P.nitems;
  if (P.band && P.nstripes <= 1 && P.i1 > P.i0) {
    const int grid = std::min(P.i1 - P.i0, P.band_grid);
    const size_t sm = band_smem_bytes(P.stage_own, P.stage_other);
    if (P.dec_dbg) k_sweep_band<true><<<grid, kBandThreads, sm, L.stream>>>(A);
    else k_sweep_band<false><<<grid, kBandThreads, sm, L.stream>>>(A);
    ++*L.counter;
    return;
  }
  const int v = (P.percell ? 4 : 0) | (P.dec_dbg != nullptr ? 2 : 0) | (P.flat ? 1 : 0);
  const dim3 g(P.nblocks), b(kSweepThreads);
  switch (v) {
    case 0: launch_pdl(k_sweep_pass<false, false, false>, g, b, 0, L.stream, A); break;
    case 1: launch_pdl(k_sweep_flat<false, false, 7>, g, b, 0, L.stream, A); break;
    case 2: launch_pdl(k_sweep_pass<false, true, false>, g, b, 0, L.stream, A); break;
    case 3: launch_pdl(k_sweep_flat<false, true, 7>, g, b, 0, L.stream, A); break;
    case 4: launch_pdl(k_sweep_pass<true, false, false>, g, b, 0, L.stream, A); break;
    case 5: launch_pdl(k_sweep_flat<true, false, 5>, g, b, 0, L.stream, A); break;
    case 6: launch_pdl(k_sweep_pass<true, true, false>, g, b, 0, L.stream, A); break;
    default: launch_pdl(k_sweep_flat<true, true, 5>, g, b, 0, L.stream, A); break;
  }
  ++*L.counter;
}

// Sec. II: every 100 iterations the acceptance rate of the window moves the cone
// half-angle by +-1 deg when outside 0.5 +- 0.05; the window restarts.
__global__ void k_advance(ChainState *st, int nchains, unsigned by, unsigned *sweep_base,
                          int adapt_now, int adapt, float tmin, float tmax) {
  pdl_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) *sweep_base += by;
  if (c >= nchains || !adapt_now) return;
  ChainState &s = st[c];
  if (adapt && s.win_att > 0) {
    const double rate = (double)s.win_acc / (double)s.win_att;
    float th = s.theta_deg;
    if (rate > 0.55) th += 1.f;
    else if (rate < 0.45) th -= 1.f;
    th = fminf(fmaxf(th, tmin), tmax);
    s.theta_deg = th;
    s.omc = 1.f - cospif(th / 180.f);
  }
  s.last_acc = s.win_acc;
  s.last_att = s.win_att;
  s.win_acc = 0;
  s.win_att = 0;
}

void launch_advance(const Launch &L, ChainState *st, int nchains, unsigned by, unsigned *sweep_base,
                    int adapt_now, int adapt, float tmin, float tmax) {
  const int nb = (nchains + 127) / 128;
  launch_pdl(k_advance, nb, 128, 0, L.stream, st, nchains, by, sweep_base, adapt_now, adapt, tmin, tmax);
  ++*L.counter;
}

}  // namespace mmc
