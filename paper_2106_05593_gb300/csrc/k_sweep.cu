// Sublattice pass of the MMC iteration (Sec. II) on all chains of a batch.
//
// Data layout (per chain): m is stored split by checkerboard colour.  Colour c
// of row r = j + ny*k holds the cells i = 2 s + ((j + k + c) & 1), s in
// [0, hx), hx = (nx + 1) / 2, as float4 (mx, my, mz, grain id) at
// m_off + c * nrows * hx + r * hx + s.  The neighbours of a colour-c cell are all
// in the other colour's array: the in-row ones at slots s - 1 + p and s + p
// (p = (j + k + c) & 1), the ones in rows j +- 1 and planes k +- 1 at slot s.
// One thread updates one cell; a block covers 256 consecutive slots of one
// chain, so a launch covers every chain of the batch.
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

namespace mmc {

struct SweepArgs {
  const ChainDev *chains;
  ChainState *st;
  const int *blk_chain;
  const long long *blk_first;
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
};

// error-free product and sum (FP32 building blocks of the length difference)
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <bool PERCELL, bool DEBUG>
__global__ void __launch_bounds__(kSweepBlock, 4) k_sweep_pass(SweepArgs A) {
  const int blk = A.blk_base + (int)blockIdx.x;
  const int c = A.blk_chain[blk];
  const ChainDev &ch = A.chains[c];
  const int nx = ch.nx, ny = ch.ny, nz = ch.nz, hx = ch.hx, nrows = ch.nrows;
  // a chain has fewer than 2^31 cells: 32-bit slot arithmetic
  const unsigned S32 = (unsigned)nrows * (unsigned)hx;
  const long long S = (long long)S32;
  const unsigned q32 = (unsigned)(blk - (int)A.blk_first[c]) * (unsigned)kSweepBlock + threadIdx.x;
  const long long q = (long long)q32;
  const int color = A.color;
  bool valid = q32 < S32;
  const int row = valid ? (int)divq(q32, ch.hx_m, ch.hx_l) : 0;
  const int s = (int)(q32 - (unsigned)row * (unsigned)hx);
  const int k = (int)divq((unsigned)row, ch.ny_m, ch.ny_l), j = row - k * ny;
  const int p = (j + k + color) & 1;
  const int i = 2 * s + p;
  valid = valid && (i < nx);
  int accepted = 0;

  if (valid) {
    const int flags = ch.flags;
    float4 *mc = A.m + ch.m_off + (long long)color * S;
    const float4 *mo = A.m + ch.m_off + (long long)(1 - color) * S;
    const float4 a = mc[q];

    // neighbours (other colour); absent bonds have weight 0
    const int pbc = ch.pbc;
    float4 nb[6];
    float w[6];
    {
      const int im = i > 0 ? i - 1 : ((pbc & 1) ? nx - 1 : -1);
      const int ip = i < nx - 1 ? i + 1 : ((pbc & 1) ? 0 : -1);
      const int jm = j > 0 ? j - 1 : ((pbc & 2) ? ny - 1 : -1);
      const int jp = j < ny - 1 ? j + 1 : ((pbc & 2) ? 0 : -1);
      const int km = k > 0 ? k - 1 : ((pbc & 4) ? nz - 1 : -1);
      const int kp = k < nz - 1 ? k + 1 : ((pbc & 4) ? 0 : -1);
      const long long rb = (long long)row * hx;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      nb[0] = im >= 0 ? mo[rb + ((im - 1 + p) >> 1)] : z4;
      nb[1] = ip >= 0 ? mo[rb + ((ip - 1 + p) >> 1)] : z4;
      nb[2] = jm >= 0 ? mo[(long long)(jm + ny * k) * hx + s] : z4;
      nb[3] = jp >= 0 ? mo[(long long)(jp + ny * k) * hx + s] : z4;
      nb[4] = km >= 0 ? mo[(long long)(j + ny * km) * hx + s] : z4;
      nb[5] = kp >= 0 ? mo[(long long)(j + ny * kp) * hx + s] : z4;
      w[0] = im >= 0 ? 1.f : 0.f;
      w[1] = ip >= 0 ? 1.f : 0.f;
      w[2] = jm >= 0 ? 1.f : 0.f;
      w[3] = jp >= 0 ? 1.f : 0.f;
      w[4] = km >= 0 ? 1.f : 0.f;
      w[5] = kp >= 0 ? 1.f : 0.f;
      if (flags & F_GRAIN) {
        const float gs = ch.gscale;
#pragma unroll
        for (int b = 0; b < 6; ++b)
          if (nb[b].w != a.w) w[b] *= gs;
      }
    }

    // material constants of this cell (kT units)
    float p2, p4, me2h, me2l, sigma, zee, k1, k2, ex, ey, ez, bs;
    if (PERCELL) {
      const float4 *tb = A.tab + ch.t_off;
      const long long off = (long long)color * S + q;
      const float4 t0 = tb[off], t1 = tb[2 * S + off], t2 = tb[4 * S + off];
      p2 = t0.x; p4 = t0.y; me2h = t0.z; me2l = 0.f; sigma = t0.w;
      zee = t1.x; k1 = t1.y; k2 = t1.z; bs = t1.w;
      ex = t2.x; ey = t2.y; ez = t2.z;
    } else {
      p2 = ch.p2; p4 = ch.p4; sigma = ch.sigma; zee = ch.zee; k1 = ch.k1; k2 = ch.k2;
      ex = ch.ex; ey = ch.ey; ez = ch.ez; bs = 1.f;
      me2h = ch.me2h; me2l = ch.me2l;
    }
    const float wx = ch.wx * bs, wy = ch.wy * bs, wz = ch.wz * bs;
    const float cdx = ch.cdx * bs, cdy = ch.cdy * bs;

    // static field: h = zee (B + mu0 H_d), kT per unit m
    float hxs, hys, hzs;
    if (flags & F_DEMAG) {
      const float4 h = A.heff[ch.h_off + (long long)color * S + q];
      hxs = h.x; hys = h.y; hzs = h.z;
    } else {
      hxs = zee * ch.Bx; hys = zee * ch.By; hzs = zee * ch.Bz;
    }

    // random numbers
    const unsigned cell = (unsigned)i + (unsigned)nx * (unsigned)row;
    const unsigned sweep = *A.sweep_base + A.sweep_off;
    const uint4 r = philox4x32_10(make_uint4(cell, sweep, (unsigned)ch.chain, 0u),
                                  make_uint2(A.key0, A.key1));
    const float u0 = uniform01(r.x), u1 = uniform01(r.y), u2 = uniform01(r.z), u3 = uniform01(r.w);

    // current length, with |m|^2 - m_e^2 kept to ~2^-48 (error-free sums)
    float xx, exx, yy, eyy, zz, ezz;
    two_prod(a.x, a.x, xx, exx);
    two_prod(a.y, a.y, yy, eyy);
    two_prod(a.z, a.z, zz, ezz);
    float s1, e1, s2, e2;
    two_sum(xx, yy, s1, e1);
    two_sum(s1, zz, s2, e2);
    const float len2 = s2;
    const float len2_lo = (e1 + e2) + (exx + eyy + ezz);
    float dh, de;
    two_sum(len2, -me2h, dh, de);
    const float delta = dh + (de + (len2_lo - me2l));    // |m|^2 - m_e^2
    const float inv = rsqrtf(len2);
    const float len = len2 * inv;
    const float n0 = a.x * inv, n1 = a.y * inv, n2 = a.z * inv;

    // orthonormal basis about n (Duff et al., JCGT 6(1), 2017)
    const float sg = n2 >= 0.f ? 1.f : -1.f;
    const float aa = -__frcp_rn(sg + n2);
    const float bb = n0 * n1 * aa;
    const float e1x = 1.f + sg * n0 * n0 * aa, e1y = sg * bb, e1z = -sg * n0;
    const float e2x = bb, e2y = sg + n1 * n1 * aa, e2z = -n1;

    // cone rotation and length change
    const float omc = A.omc_override >= 0.f ? A.omc_override : A.st[c].omc;
    const float t = u0 * omc;
    const float ct = 1.f - t;
    const float st = sqrtf(t * (2.f - t));
    float sp, cp;
    sincospif(2.f * u1, &sp, &cp);
    const float dx = ct * n0 + st * (cp * e1x + sp * e2x);
    const float dy = ct * n1 + st * (cp * e1y + sp * e2y);
    const float dz = ct * n2 + st * (cp * e1z + sp * e2z);
    const float tt = sigma * (2.f * u2 - 1.f);
    const float ls = len * (1.f + tt);
    const float mpx = ls * dx, mpy = ls * dy, mpz = ls * dz;
    const float dmx = mpx - a.x, dmy = mpy - a.y, dmz = mpz - a.z;

    // exchange: sum_j w_j (|m' - m_j|^2 - |m - m_j|^2) = sum_j w_j dm.(m' + m - 2 m_j)
    const float wd[6] = {wx, wx, wy, wy, wz, wz};
    float fex = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float vx = (mpx - nb[b].x) + (a.x - nb[b].x);
      const float vy = (mpy - nb[b].y) + (a.y - nb[b].y);
      const float vz = (mpz - nb[b].z) + (a.z - nb[b].z);
      fex = fmaf(wd[b] * w[b], dmx * vx + dmy * vy + dmz * vz, fex);
    }
    if (nz > 1) {
#pragma unroll
      for (int b = 4; b < 6; ++b) {
        const float vx = (mpx - nb[b].x) + (a.x - nb[b].x);
        const float vy = (mpy - nb[b].y) + (a.y - nb[b].y);
        const float vz = (mpz - nb[b].z) + (a.z - nb[b].z);
        fex = fmaf(wd[b] * w[b], dmx * vx + dmy * vy + dmz * vz, fex);
      }
    }
    // interfacial DMI: linear in m_i
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (flags & F_DMI) {
      gx = cdx * (w[1] * nb[1].z - w[0] * nb[0].z);
      gy = cdy * (w[3] * nb[3].z - w[2] * nb[2].z);
      gz = -cdx * (w[1] * nb[1].x - w[0] * nb[0].x) - cdy * (w[3] * nb[3].y - w[2] * nb[2].y);
    }
    const float flin = dmx * (gx - hxs) + dmy * (gy - hys) + dmz * (gz - hzs);

    // longitudinal (Eq. 7): dq = m'^2 - m^2 = m^2 t (2 + t)
    const float dq = len2 * tt * (2.f + tt);
    const float flong = dq * (p2 + p4 * (2.f * delta + dq));

    // anisotropy
    float fan = 0.f;
    if (flags & F_CUBIC) {
      const float a2 = n0 * n0, b2 = n1 * n1, c2 = n2 * n2;
      const float A2 = dx * dx, B2 = dy * dy, C2 = dz * dz;
      const float eo = k1 * (a2 * b2 + a2 * c2 + b2 * c2) + k2 * a2 * b2 * c2;
      const float en = k1 * (A2 * B2 + A2 * C2 + B2 * C2) + k2 * A2 * B2 * C2;
      fan = en - eo;
    } else if (flags & F_ANIS) {
      const float ca = n0 * ex + n1 * ey + n2 * ez;
      const float cb = dx * ex + dy * ey + dz * ez;
      const float dd = (ca - cb) * (ca + cb);
      fan = dd * (k1 + k2 * (2.f - ca * ca - cb * cb));
    }

    const float dF = fex + flin + flong + fan;
    // ln(1 + t): Taylor series through t^7 when |t| <= 0.05 (error below t^8 / 8)
    float lg;
    if (fabsf(tt) <= 0.05f)
      lg = tt * (1.f - tt * (0.5f - tt * (1.f / 3.f - tt * (0.25f - tt * (0.2f - tt * (1.f / 6.f - tt * (1.f / 7.f)))))));
    else
      lg = log1pf(tt);
    const float dl = dF - 4.f * lg;
    // ln u3 < 0: a non-positive dl accepts whatever u3 is, so its log is skipped
    float dec;
    if (DEBUG || dl > 0.f) dec = dl + logf(u3);
    else dec = dl;
    accepted = dec < 0.f;
    if (accepted) mc[q] = make_float4(mpx, mpy, mpz, a.w);
    if (DEBUG) {
      A.dec_dbg[cell] = dec;
      A.acc_dbg[cell] = (signed char)accepted;
    }
  }

  // acceptance counts: warp ballots, then one atomic per block
  __shared__ unsigned wacc[kSweepBlock / 32], watt[kSweepBlock / 32];
  const unsigned ba = __ballot_sync(0xffffffffu, accepted);
  const unsigned bv = __ballot_sync(0xffffffffu, valid);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    wacc[warp] = __popc(ba);
    watt[warp] = __popc(bv);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned sa = 0, sv = 0;
#pragma unroll
    for (int w2 = 0; w2 < kSweepBlock / 32; ++w2) { sa += wacc[w2]; sv += watt[w2]; }
    if (sv) {
      atomicAdd(&A.st[c].win_acc, (unsigned long long)sa);
      atomicAdd(&A.st[c].win_att, (unsigned long long)sv);
    }
  }
}

void launch_sweep_pass(const Launch &L, const SweepLaunch &P) {
  SweepArgs A;
  A.chains = P.chains; A.st = P.st; A.blk_chain = P.blk_chain; A.blk_first = P.blk_first;
  A.blk_base = P.blk_base;
  A.m = P.m; A.heff = P.heff; A.tab = P.tab; A.sweep_base = P.sweep_base;
  A.sweep_off = P.sweep_off; A.key0 = P.key0; A.key1 = P.key1; A.color = P.color;
  A.omc_override = P.omc_override; A.dec_dbg = P.dec_dbg; A.acc_dbg = P.acc_dbg;
  const bool dbg = P.dec_dbg != nullptr;
  if (P.percell) {
    if (dbg) k_sweep_pass<true, true><<<P.nblocks, kSweepBlock, 0, L.stream>>>(A);
    else k_sweep_pass<true, false><<<P.nblocks, kSweepBlock, 0, L.stream>>>(A);
  } else {
    if (dbg) k_sweep_pass<false, true><<<P.nblocks, kSweepBlock, 0, L.stream>>>(A);
    else k_sweep_pass<false, false><<<P.nblocks, kSweepBlock, 0, L.stream>>>(A);
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
