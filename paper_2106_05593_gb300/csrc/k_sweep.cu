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
#include <cstdio>

#include "mmc_internal.h"
#include "philox.cuh"
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
  const int2 bd = A.blk_desc[A.blk_base + (int)blockIdx.x];
  const int c = bd.x;
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
      a[e] = mc[q32];
      load_neighbours(pbc, (flags & F_GRAIN) != 0, K.gscale, nx, ny, nz, hx, mo, a[e], i, j, k, row, s, p, nb[e], w[e]);
      M[e] = cell_material<PERCELL>(K, A.tab, S, (long long)color * S + q32);
      if (flags & F_DEMAG) h[e] = A.heff[K.h_off + (long long)color * S + q32];
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
    if (accepted[e]) mc[qq[e]] = make_float4(v.mpx, v.mpy, v.mpz, a[e].w);
    if (DEBUG) {
      A.dec_dbg[cellid[e]] = dec;
      A.acc_dbg[cellid[e]] = (signed char)accepted[e];
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

void launch_sweep_pass(const Launch &L, const SweepLaunch &P) {
  SweepArgs A;
  A.chains = P.chains; A.st = P.st; A.blk_desc = P.blk_desc;
  A.blk_base = P.blk_base;
  A.m = P.m; A.heff = P.heff; A.tab = P.tab; A.sweep_base = P.sweep_base;
  A.sweep_off = P.sweep_off; A.key0 = P.key0; A.key1 = P.key1; A.color = P.color;
  A.omc_override = P.omc_override; A.dec_dbg = P.dec_dbg; A.acc_dbg = P.acc_dbg;
  A.nstripes = P.nstripes; A.stripe = P.stripe;
  const int v = (P.percell ? 4 : 0) | (P.dec_dbg != nullptr ? 2 : 0) | (P.flat ? 1 : 0);
  switch (v) {
    case 0: k_sweep_pass<false, false, false><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
    case 1: k_sweep_pass<false, false, true><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
    case 2: k_sweep_pass<false, true, false><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
    case 3: k_sweep_pass<false, true, true><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
    case 4: k_sweep_pass<true, false, false><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
    case 5: k_sweep_pass<true, false, true><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
    case 6: k_sweep_pass<true, true, false><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
    default: k_sweep_pass<true, true, true><<<P.nblocks, kSweepThreads, 0, L.stream>>>(A); break;
  }
  ++*L.counter;
}

// Sec. II: every 100 iterations the acceptance rate of the window moves the cone
// half-angle by +-1 deg when outside 0.5 +- 0.05; the window restarts.
__global__ void k_advance(ChainState *st, int nchains, unsigned by, unsigned *sweep_base,
                          int adapt_now, int adapt, float tmin, float tmax) {
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
  k_advance<<<nb, 128, 0, L.stream>>>(st, nchains, by, sweep_base, adapt_now, adapt, tmin, tmax);
  ++*L.counter;
}

}  // namespace mmc
