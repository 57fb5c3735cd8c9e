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
  unsigned rk[20];          // Philox round keys of (key0, key1), see philox4x32_10_rk
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

// One-cell-thick chains (every chain of the launch has nz = 1): the same pass
// with the work per cell cut down.  The chain constants are read once per block
// into shared memory; the Philox round keys come precomputed in the kernel
// parameters; the four in-plane neighbours are found by offsets from the cell's
// slot in the other colour (s - 1 + p, s + p in the row, s in the rows j -+ 1,
// with the periodic wrap at the edges); exchange, DMI and the field act through
// one local vector (local_change_flat).
template <bool PERCELL, bool DEBUG, int MINB>
__global__ void __launch_bounds__(kSweepThreads, MINB) k_sweep_flat(SweepArgs A) {
  __shared__ float4 skv[kChainKVec];
  __shared__ unsigned wacc[kSweepThreads / 32], watt[kSweepThreads / 32];
  const int2 bd = A.blk_desc[A.blk_base + (int)blockIdx.x];
  const int c = bd.x;
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
      a[e] = mc[q32];
      // the other colour's slots of the -x, +x, -y, +y neighbours, relative to
      // slot s of row j (periodic axes have even extents)
      const float4 *P = mo + (long long)j * hx + s;
      const bool hl = i > 0 || (pbc & 1), hr = i < nx - 1 || (pbc & 1);
      const bool hu = j > 0 || (pbc & 2), hd = j < ny - 1 || (pbc & 2);
      const int ol = i > 0 ? p - 1 : hx - 1;
      const int orr = i < nx - 1 ? p : 1 - hx;
      const int ou = j > 0 ? -hx : (ny - 1) * hx;
      const int od = j < ny - 1 ? hx : -(ny - 1) * hx;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      nb[e][0] = hl ? P[ol] : z4;
      nb[e][1] = hr ? P[orr] : z4;
      nb[e][2] = hu ? P[ou] : z4;
      nb[e][3] = hd ? P[od] : z4;
      pres[e][0] = hl ? 1.f : 0.f;
      pres[e][1] = hr ? 1.f : 0.f;
      pres[e][2] = hu ? 1.f : 0.f;
      pres[e][3] = hd ? 1.f : 0.f;
      if (grain) {
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (nb[e][b].w != a[e].w) pres[e][b] *= K.gscale;
      }
      M[e] = cell_material<PERCELL>(K, A.tab, S, (long long)color * S + q32);
      if (flags & F_DEMAG) h[e] = A.heff[K.h_off + (long long)color * S + q32];
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
    lgv[e] = log1p_move(ga[e].tt);
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
  {
    unsigned k0 = P.key0, k1 = P.key1;
    for (int r = 0; r < 10; ++r) {
      A.rk[2 * r] = k0;
      A.rk[2 * r + 1] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
  const int v = (P.percell ? 4 : 0) | (P.dec_dbg != nullptr ? 2 : 0) | (P.flat ? 1 : 0);
  const dim3 g(P.nblocks), b(kSweepThreads);
  switch (v) {
    case 0: k_sweep_pass<false, false, false><<<g, b, 0, L.stream>>>(A); break;
    case 1:
      // the production pass of uniform one-cell-thick chains comes in three
      // occupancies (blocks per SM), picked by timing at create
      if (P.variant == 1) k_sweep_flat<false, false, 6><<<g, b, 0, L.stream>>>(A);
      else if (P.variant == 2) k_sweep_flat<false, false, 7><<<g, b, 0, L.stream>>>(A);
      else k_sweep_flat<false, false, 8><<<g, b, 0, L.stream>>>(A);
      break;
    case 2: k_sweep_pass<false, true, false><<<g, b, 0, L.stream>>>(A); break;
    case 3: k_sweep_flat<false, true, 8><<<g, b, 0, L.stream>>>(A); break;
    case 4: k_sweep_pass<true, false, false><<<g, b, 0, L.stream>>>(A); break;
    case 5: k_sweep_flat<true, false, 5><<<g, b, 0, L.stream>>>(A); break;
    case 6: k_sweep_pass<true, true, false><<<g, b, 0, L.stream>>>(A); break;
    default: k_sweep_flat<true, true, 5><<<g, b, 0, L.stream>>>(A); break;
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
