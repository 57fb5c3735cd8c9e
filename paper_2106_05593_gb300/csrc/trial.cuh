// Per-cell pieces of the MMC trial move (Sec. II), shared by the sublattice
// pass (k_sweep.cu) and the serial exact-demag sweep (k_serial.cu).  All
// energies are in units of kT.
#pragma once

#include "mmc_internal.h"

namespace mmc {

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

// chain constants a trial needs, loaded from the first 176 bytes of ChainDev
// as eleven 16-byte vectors (one load instruction each instead of one per field)
struct ChainK {
  int nx, ny, nz, hx, nrows, pbc, flags, chain;
  unsigned hx_m, ny_m;
  int hx_l, ny_l;
  float gscale, wx, wy, wz, cdx, cdy, p2, p4, me2h, me2l, sigma, zee, k1, k2, ex, ey, ez, Bx, By, Bz, Ms0;
  long long m_off, h_off, t_off, ms_off;
};

constexpr int kChainKVec = 11;     // 16-byte vectors of ChainDev that ChainK unpacks

__device__ __forceinline__ ChainK load_chain(const ChainDev *cd) {
  const int4 *iv = reinterpret_cast<const int4 *>(cd);
  const float4 *fv = reinterpret_cast<const float4 *>(cd);
  const longlong2 *lv = reinterpret_cast<const longlong2 *>(cd);
  const int4 a = iv[0], b = iv[1], u = iv[2], l = iv[3];
  const float4 f0 = fv[4], f1 = fv[5], f2 = fv[6], f3 = fv[7], f4 = fv[8];
  const longlong2 o0 = lv[9], o1 = lv[10];
  ChainK K;
  K.nx = a.x; K.ny = a.y; K.nz = a.z; K.hx = a.w;
  K.nrows = b.x; K.pbc = b.y; K.flags = b.z; K.chain = b.w;
  K.hx_m = (unsigned)u.x; K.ny_m = (unsigned)u.y;
  K.hx_l = l.x; K.ny_l = l.y; K.gscale = __int_as_float(l.w);
  K.wx = f0.x; K.wy = f0.y; K.wz = f0.z; K.cdx = f0.w;
  K.cdy = f1.x; K.p2 = f1.y; K.p4 = f1.z; K.me2h = f1.w;
  K.me2l = f2.x; K.sigma = f2.y; K.zee = f2.z; K.k1 = f2.w;
  K.k2 = f3.x; K.ex = f3.y; K.ey = f3.z; K.ez = f3.w;
  K.Bx = f4.x; K.By = f4.y; K.Bz = f4.z; K.Ms0 = f4.w;
  K.m_off = o0.x; K.h_off = o0.y; K.t_off = o1.x; K.ms_off = o1.y;
  return K;
}

// a chain's constants from a copy of its first kChainKVec vectors (shared memory)
__device__ __forceinline__ ChainK load_chain_vec(const float4 *v) {
  return load_chain(reinterpret_cast<const ChainDev *>(v));
}

// material constants of one cell
struct CellMat {
  float p2, p4, me2h, me2l, sigma, zee, k1, k2, ex, ey, ez, bs;
};

// off = colour * S + slot; per-cell tables are 3 float4 arrays of 2 S entries:
// {p2, p4, m_e^2 (high part), sigma}, {zee, k1, k2, bond scale}, {e_A, m_e^2 low part}
template <bool PERCELL, typename CH>
__device__ __forceinline__ CellMat cell_material(const CH &ch, const float4 *tab, long long S, long long off,
                                                 MmcCheck *ck = nullptr) {
  CellMat M;
  if (PERCELL) {
    const float4 *tb = tab + ch.t_off;
    off = MMC_CK(ck, off, 0, 2 * S, kCkSweepTable);
    const float4 t0 = tb[off], t1 = tb[2 * S + off], t2 = tb[4 * S + off];
    M.p2 = t0.x; M.p4 = t0.y; M.me2h = t0.z; M.me2l = t2.w; M.sigma = t0.w;
    M.zee = t1.x; M.k1 = t1.y; M.k2 = t1.z; M.bs = t1.w;
    M.ex = t2.x; M.ey = t2.y; M.ez = t2.z;
  } else {
    M.p2 = ch.p2; M.p4 = ch.p4; M.sigma = ch.sigma; M.zee = ch.zee; M.k1 = ch.k1; M.k2 = ch.k2;
    M.ex = ch.ex; M.ey = ch.ey; M.ez = ch.ez; M.bs = 1.f;
    M.me2h = ch.me2h; M.me2l = ch.me2l;
  }
  return M;
}

// the six neighbours of cell (i, j, k) of colour `color`, all in the other
// colour's array mo; absent bonds get weight 0, bonds across grains gscale
__device__ __forceinline__ void load_neighbours(int pbc, bool grain, float gscale, int nx, int ny, int nz, int hx,
                                                const float4 *mo, float4 a, int i, int j, int k, int row, int s,
                                                int p, float4 nb[6], float w[6], MmcCheck *ck = nullptr,
                                                long long S = 0) {
  const int im = i > 0 ? i - 1 : ((pbc & 1) ? nx - 1 : -1);
  const int ip = i < nx - 1 ? i + 1 : ((pbc & 1) ? 0 : -1);
  const int jm = j > 0 ? j - 1 : ((pbc & 2) ? ny - 1 : -1);
  const int jp = j < ny - 1 ? j + 1 : ((pbc & 2) ? 0 : -1);
  const int km = k > 0 ? k - 1 : ((pbc & 4) ? nz - 1 : -1);
  const int kp = k < nz - 1 ? k + 1 : ((pbc & 4) ? 0 : -1);
  const long long rb = (long long)row * hx;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  nb[0] = im >= 0 ? mo[MMC_CK(ck, rb + ((im - 1 + p) >> 1), 0, S, kCkSweepNeighbour)] : z4;
  nb[1] = ip >= 0 ? mo[MMC_CK(ck, rb + ((ip - 1 + p) >> 1), 0, S, kCkSweepNeighbour)] : z4;
  nb[2] = jm >= 0 ? mo[MMC_CK(ck, (long long)(jm + ny * k) * hx + s, 0, S, kCkSweepNeighbour)] : z4;
  nb[3] = jp >= 0 ? mo[MMC_CK(ck, (long long)(jp + ny * k) * hx + s, 0, S, kCkSweepNeighbour)] : z4;
  nb[4] = km >= 0 ? mo[MMC_CK(ck, (long long)(j + ny * km) * hx + s, 0, S, kCkSweepNeighbour)] : z4;
  nb[5] = kp >= 0 ? mo[MMC_CK(ck, (long long)(j + ny * kp) * hx + s, 0, S, kCkSweepNeighbour)] : z4;
  w[0] = im >= 0 ? 1.f : 0.f;
  w[1] = ip >= 0 ? 1.f : 0.f;
  w[2] = jm >= 0 ? 1.f : 0.f;
  w[3] = jp >= 0 ? 1.f : 0.f;
  w[4] = km >= 0 ? 1.f : 0.f;
  w[5] = kp >= 0 ? 1.f : 0.f;
  if (grain) {
#pragma unroll
    for (int b = 0; b < 6; ++b)
      if (nb[b].w != a.w) w[b] *= gscale;
  }
}

// sin(pi x) and cos(pi x) for x in [0, 2]: x = n / 2 + r with n = rint(2 x) and
// |r| <= 1/4 (r exact), sin and cos of t = pi r from their Taylor series through
// t^9 and t^10 (|t| <= pi / 4: truncation below 2e-9), then the rotation by
// n quarter turns.
__device__ __forceinline__ void sincospi_move(float x, float &s, float &c) {
  const float n = rintf(2.f * x);
  const float r = fmaf(-0.5f, n, x);
  const float t = 3.14159265358979323846f * r;
  const float t2 = t * t;
  // 1/3!, 1/5!, 1/7!, 1/9!  and  1/2!, 1/4!, 1/6!, 1/8!, 1/10!
  const float sr = t * fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 2.7557319224e-6f, -1.9841269841e-4f),
                                               8.3333333333e-3f), -1.6666666667e-1f), 1.f);
  const float cr = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, -2.7557319224e-7f, 2.4801587302e-5f),
                                                    -1.3888888889e-3f), 4.1666666667e-2f), -0.5f), 1.f);
  const int q = (int)n & 3;
  const float a = (q & 1) ? cr : sr, b = (q & 1) ? sr : cr;
  s = (q & 2) ? -a : a;
  c = ((q + 1) & 2) ? -b : b;
}

// The move: a rotation uniform on the cap of half-angle theta about m/|m|
// (cos = 1 - u0 (1 - cos theta), phi = 2 pi u1, orthonormal basis of Duff et
// al., JCGT 6(1), 2017) times the length factor 1 + sigma (2 u2 - 1).
struct Move {
  float len2, delta;         // |m|^2 and |m|^2 - m_e^2 (the latter to ~2^-48)
  float len;                 // |m|
  float n0, n1, n2;          // m / |m|
  float dx, dy, dz;          // new direction
  float tt;                  // sigma (2 u2 - 1)
  float mpx, mpy, mpz;       // m'
  float dmx, dmy, dmz;       // m' - m
};

// first half: the current length and direction
__device__ __forceinline__ Move move_length(float4 a, float me2h, float me2l) {
  Move v;
  float xx, exx, yy, eyy, zz, ezz;
  two_prod(a.x, a.x, xx, exx);
  two_prod(a.y, a.y, yy, eyy);
  two_prod(a.z, a.z, zz, ezz);
  float s1, e1, s2, e2;
  two_sum(xx, yy, s1, e1);
  two_sum(s1, zz, s2, e2);
  v.len2 = s2;
  const float len2_lo = (e1 + e2) + (exx + eyy + ezz);
  float dh, de;
  two_sum(v.len2, -me2h, dh, de);
  v.delta = dh + (de + (len2_lo - me2l));
  const float inv = rsqrtf(v.len2);
  v.len = v.len2 * inv;
  v.n0 = a.x * inv; v.n1 = a.y * inv; v.n2 = a.z * inv;
  return v;
}

// second half: the proposed moment m'
__device__ __forceinline__ void move_direction(Move &v, float4 a, float sigma, float omc, float u0, float u1,
                                               float u2) {
  const float sg = v.n2 >= 0.f ? 1.f : -1.f;
  const float aa = -__fdividef(1.f, sg + v.n2);     // |sg + n2| >= 1
  const float bb = v.n0 * v.n1 * aa;
  const float e1x = 1.f + sg * v.n0 * v.n0 * aa, e1y = sg * bb, e1z = -sg * v.n0;
  const float e2x = bb, e2y = sg + v.n1 * v.n1 * aa, e2z = -v.n1;

  const float t = u0 * omc;
  const float ct = 1.f - t;
  const float t2 = t * (2.f - t);                  // > 0: t = u0 (1 - cos theta) in (0, 2)
  const float st = t2 * rsqrtf(t2);
  float sp, cp;
  sincospi_move(2.f * u1, sp, cp);
  v.dx = ct * v.n0 + st * (cp * e1x + sp * e2x);
  v.dy = ct * v.n1 + st * (cp * e1y + sp * e2y);
  v.dz = ct * v.n2 + st * (cp * e1z + sp * e2z);
  v.tt = sigma * (2.f * u2 - 1.f);
  const float ls = v.len * (1.f + v.tt);
  v.mpx = ls * v.dx; v.mpy = ls * v.dy; v.mpz = ls * v.dz;
  v.dmx = v.mpx - a.x; v.dmy = v.mpy - a.y; v.dmz = v.mpz - a.z;
}

// The parts of a move that depend only on its random numbers, not on m: the
// cone's cos / sin, the azimuth's cos / sin and the length factor (the same
// operations as move_direction), so that they can run while m is being loaded.
struct MoveAngles {
  float ct, st, cp, sp, tt;
};
__device__ __forceinline__ MoveAngles move_angles(float sigma, float omc, float u0, float u1, float u2) {
  MoveAngles g;
  const float t = u0 * omc;
  g.ct = 1.f - t;
  const float t2 = t * (2.f - t);
  g.st = t2 * rsqrtf(t2);
  sincospi_move(2.f * u1, g.sp, g.cp);
  g.tt = sigma * (2.f * u2 - 1.f);
  return g;
}
// move_direction with the angles given
__device__ __forceinline__ void move_direction_g(Move &v, float4 a, const MoveAngles &g) {
  const float sg = v.n2 >= 0.f ? 1.f : -1.f;
  const float aa = -__fdividef(1.f, sg + v.n2);
  const float bb = v.n0 * v.n1 * aa;
  const float e1x = 1.f + sg * v.n0 * v.n0 * aa, e1y = sg * bb, e1z = -sg * v.n0;
  const float e2x = bb, e2y = sg + v.n1 * v.n1 * aa, e2z = -v.n1;
  v.dx = g.ct * v.n0 + g.st * (g.cp * e1x + g.sp * e2x);
  v.dy = g.ct * v.n1 + g.st * (g.cp * e1y + g.sp * e2y);
  v.dz = g.ct * v.n2 + g.st * (g.cp * e1z + g.sp * e2z);
  v.tt = g.tt;
  const float ls = v.len * (1.f + v.tt);
  v.mpx = ls * v.dx; v.mpy = ls * v.dy; v.mpz = ls * v.dz;
  v.dmx = v.mpx - a.x; v.dmy = v.mpy - a.y; v.dmz = v.mpz - a.z;
}

// exchange (pair form of Eq. 10): sum_j w_j (|m' - m_j|^2 - |m - m_j|^2)
__device__ __forceinline__ float exchange_change(const Move &v, float4 a, const float4 nb[6], const float w[6],
                                                 float wx, float wy, float wz, bool has_z) {
  const float wd[6] = {wx, wx, wy, wy, wz, wz};
  float fex = 0.f;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const float vx = (v.mpx - nb[b].x) + (a.x - nb[b].x);
    const float vy = (v.mpy - nb[b].y) + (a.y - nb[b].y);
    const float vz = (v.mpz - nb[b].z) + (a.z - nb[b].z);
    fex = fmaf(wd[b] * w[b], v.dmx * vx + v.dmy * vy + v.dmz * vz, fex);
  }
  if (has_z) {
#pragma unroll
    for (int b = 4; b < 6; ++b) {
      const float vx = (v.mpx - nb[b].x) + (a.x - nb[b].x);
      const float vy = (v.mpy - nb[b].y) + (a.y - nb[b].y);
      const float vz = (v.mpz - nb[b].z) + (a.z - nb[b].z);
      fex = fmaf(wd[b] * w[b], v.dmx * vx + v.dmy * vy + v.dmz * vz, fex);
    }
  }
  return fex;
}

// interfacial DMI (pair form of Eq. 15, linear in m_i) plus Zeeman and the
// frozen demag field (Eq. 14): dm . (g - h)
__device__ __forceinline__ float linear_change(const Move &v, const float4 nb[6], const float w[6], float cdx,
                                               float cdy, bool dmi, float hxs, float hys, float hzs) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (dmi) {
    gx = cdx * (w[1] * nb[1].z - w[0] * nb[0].z);
    gy = cdy * (w[3] * nb[3].z - w[2] * nb[2].z);
    gz = -cdx * (w[1] * nb[1].x - w[0] * nb[0].x) - cdy * (w[3] * nb[3].y - w[2] * nb[2].y);
  }
  return v.dmx * (gx - hxs) + v.dmy * (gy - hys) + v.dmz * (gz - hzs);
}

// exchange (pair form of Eq. 10), interfacial DMI (pair form of Eq. 15) and the
// Zeeman + frozen demag field (Eq. 14) of a cell of a one-cell-thick chain, as
// one product dm . u: the exchange change sum_b w_b (|m' - m_b|^2 - |m - m_b|^2)
// is sum_b w_b dm . (m' + m - 2 m_b); nb[0..3] are the -x, +x, -y, +y
// neighbours, w[b] their full bond weights (0 for an absent bond), d[b] their
// DMI presence weights, h the field term (kT per unit m).
__device__ __forceinline__ float local_change_flat(const Move &v, float4 a, const float4 nb[4], const float w[4],
                                                   const float d[4], float cdx, float cdy, bool dmi, float hx,
                                                   float hy, float hz) {
  const float sx = v.mpx + a.x, sy = v.mpy + a.y, sz = v.mpz + a.z;
  float ux = -hx, uy = -hy, uz = -hz;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    ux = fmaf(w[b], fmaf(-2.f, nb[b].x, sx), ux);
    uy = fmaf(w[b], fmaf(-2.f, nb[b].y, sy), uy);
    uz = fmaf(w[b], fmaf(-2.f, nb[b].z, sz), uz);
  }
  if (dmi) {
    ux = fmaf(cdx, d[1] * nb[1].z - d[0] * nb[0].z, ux);
    uy = fmaf(cdy, d[3] * nb[3].z - d[2] * nb[2].z, uy);
    uz = fmaf(-cdx, d[1] * nb[1].x - d[0] * nb[0].x, uz);
    uz = fmaf(-cdy, d[3] * nb[3].y - d[2] * nb[2].y, uz);
  }
  return v.dmx * ux + v.dmy * uy + v.dmz * uz;
}

// longitudinal term (exponent of Eq. 7): dq = m'^2 - m^2 = m^2 t (2 + t)
__device__ __forceinline__ float longitudinal_change(const Move &v, float p2, float p4) {
  const float dq = v.len2 * v.tt * (2.f + v.tt);
  return dq * (p2 + p4 * (2.f * v.delta + dq));
}

// anisotropy (Eq. 11 uniaxial, Eq. 12 cubic) on the unit directions
__device__ __forceinline__ float anisotropy_change(const Move &v, int flags, float k1, float k2, float ex, float ey,
                                                   float ez) {
  float fan = 0.f;
  if (flags & F_CUBIC) {
    const float a2 = v.n0 * v.n0, b2 = v.n1 * v.n1, c2 = v.n2 * v.n2;
    const float A2 = v.dx * v.dx, B2 = v.dy * v.dy, C2 = v.dz * v.dz;
    const float eo = k1 * (a2 * b2 + a2 * c2 + b2 * c2) + k2 * a2 * b2 * c2;
    const float en = k1 * (A2 * B2 + A2 * C2 + B2 * C2) + k2 * A2 * B2 * C2;
    fan = en - eo;
  } else if (flags & F_ANIS) {
    const float ca = v.n0 * ex + v.n1 * ey + v.n2 * ez;
    const float cb = v.dx * ex + v.dy * ey + v.dz * ez;
    const float dd = (ca - cb) * (ca + cb);
    fan = dd * (k1 + k2 * (2.f - ca * ca - cb * cb));
  }
  return fan;
}

// ln(1 + t): Taylor series through t^7 when |t| <= 0.05 (error below t^8 / 8)
__device__ __forceinline__ float log1p_series(float tt) {
  return tt * (1.f - tt * (0.5f - tt * (1.f / 3.f - tt * (0.25f - tt * (0.2f - tt * (1.f / 6.f - tt * (1.f / 7.f)))))));
}
__device__ __forceinline__ float log1p_move(float tt) {
  if (fabsf(tt) <= 0.05f) return log1p_series(tt);
  return log1pf(tt);
}
// the same for a cell of a chain whose length-move width is sigma (|t| <= sigma):
// one branch per chain instead of one per cell when sigma <= 0.05
__device__ __forceinline__ float log1p_move_s(float tt, float sigma) {
  return sigma <= 0.05f ? log1p_series(tt) : log1p_move(tt);
}

}  // namespace mmc
