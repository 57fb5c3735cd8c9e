// Differentiable energy (forward + hand-written backward) of one chain for a
// caller-given state m (natural order, 3 values per cell, float or double).
//
// Energy terms (J, FP64 sums):
//   exchange  c_ex,a |m_i - m_j|^2 per bond (Eq. 10 counts each bond twice)
//   DMI       -(V D0 / h_a) d.(m_i x m_j), d = z x e_a, in-plane bonds (Eq. 15)
//   anisotropy V [K1(T) (1 - (u.e)^2) + K2(T) (1 - (u.e)^2)^2], u = m/|m| (Eq. 11)
//   Zeeman    -V Ms0 m.B
//   longitudinal c2 |m|^2 + c4 (|m|^2 - me2)^2 (Eq. 7 exponent times kT)
//   demag     -(mu0 V / 2) Ms0 m.H_d (Eq. 14), H_d from the FFT convolution
// Gradient dE/dm_i in the precision T; the parameter gradients are assembled on
// the host from per-unit sums (dE/dA0 = sum V/h^2 |dm|^2, ...).
#include "mmc_internal.h"

namespace mmc {

template <typename T>
__device__ __forceinline__ T dsqrt(T v);
template <> __device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(v); }

template <typename T>
__global__ void __launch_bounds__(kReduceBlock)
k_energy_grad(const ChainDev *chains, int c, const T *m, const double *Hd, GradCoef G, T *dEdm,
              double *part) {
  __shared__ double red[kReduceBlock / 32][8];
  const ChainDev &ch = chains[c];
  const int nx = ch.nx, ny = ch.ny, nz = ch.nz;
  const long long n = (long long)nx * ny * nz;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // ex_unit, dmi_unit, an, an1_unit, zee, long, demag
  for (int t = 0; t < 4; ++t) {
    const long long q = (long long)blockIdx.x * kReduceBlock * 4 + t * kReduceBlock + threadIdx.x;
    if (q >= n) break;
    const int i = (int)(q % nx);
    const int j = (int)((q / nx) % ny);
    const int k = (int)(q / ((long long)nx * ny));
    const T mx = m[3 * q], my = m[3 * q + 1], mz = m[3 * q + 2];
    T gx = 0, gy = 0, gz = 0;
    const int ext[3] = {nx, ny, nz};
    const int pos[3] = {i, j, k};
    const long long stride[3] = {1, nx, (long long)nx * ny};
    for (int a = 0; a < 3; ++a) {
      for (int dir = -1; dir <= 1; dir += 2) {
        int p = pos[a] + dir;
        if (p < 0 || p >= ext[a]) {
          if (!((ch.pbc >> a) & 1)) continue;
          p = (p + ext[a]) % ext[a];
        }
        const long long r = q + (long long)(p - pos[a]) * stride[a];
        const T ux = m[3 * r], uy = m[3 * r + 1], uz = m[3 * r + 2];
        const T cex = (T)G.cex[a];
        gx += 2 * cex * (mx - ux);
        gy += 2 * cex * (my - uy);
        gz += 2 * cex * (mz - uz);
        if (dir > 0) {
          const double dx = (double)mx - ux, dy = (double)my - uy, dz = (double)mz - uz;
          acc[0] += G.vh2[a] * (dx * dx + dy * dy + dz * dz);
        }
        if (a < 2 && G.dmi) {
          const T cd = (T)G.cdmi[a];
          const T ua = a == 0 ? ux : uy;
          // linear coefficient of m_i (both bond directions)
          if (a == 0) gx += dir * cd * uz; else gy += dir * cd * uz;
          gz -= dir * cd * ua;
          if (dir > 0) {
            const double qa = a == 0 ? (double)mx : (double)my;
            acc[1] += -G.vh[a] * ((double)mz * ua - qa * (double)uz);
          }
        }
      }
    }
    // single-site terms
    const double l2 = (double)mx * mx + (double)my * my + (double)mz * mz;
    const T l2t = mx * mx + my * my + mz * mz;
    const T len = dsqrt<T>(l2t);
    if (len > 0) {
      const T u0 = mx / len, u1 = my / len, u2 = mz / len;
      if (G.cubic) {
        const T a2 = u0 * u0, b2 = u1 * u1, c2 = u2 * u2;
        const T K1 = (T)G.K1T, K2 = (T)G.K2T, V = (T)G.V;
        acc[2] += G.V * (G.K1T * ((double)a2 * b2 + (double)a2 * c2 + (double)b2 * c2) + G.K2T * (double)a2 * b2 * c2);
        acc[3] += G.V * G.Kscale * ((double)a2 * b2 + (double)a2 * c2 + (double)b2 * c2);
        T du[3] = {V * (K1 * 2 * u0 * (b2 + c2) + K2 * 2 * u0 * b2 * c2),
                   V * (K1 * 2 * u1 * (a2 + c2) + K2 * 2 * u1 * a2 * c2),
                   V * (K1 * 2 * u2 * (a2 + b2) + K2 * 2 * u2 * a2 * b2)};
        const T dot = du[0] * u0 + du[1] * u1 + du[2] * u2;
        gx += (du[0] - dot * u0) / len;
        gy += (du[1] - dot * u1) / len;
        gz += (du[2] - dot * u2) / len;
      } else if (G.anis) {
        const T e0 = (T)G.e[0], e1 = (T)G.e[1], e2 = (T)G.e[2];
        const T d = u0 * e0 + u1 * e1 + u2 * e2;
        const double dd = (double)d;
        const double sn = 1.0 - dd * dd;
        acc[2] += G.V * (G.K1T * sn + G.K2T * sn * sn);
        acc[3] += G.V * G.Kscale * sn;
        const T coef = -2 * (T)G.V * ((T)G.K1T + 2 * (T)G.K2T * (1 - d * d)) * d / len;
        gx += coef * (e0 - d * u0);
        gy += coef * (e1 - d * u1);
        gz += coef * (e2 - d * u2);
      }
    }
    acc[4] += -G.V * G.Ms0 * ((double)mx * G.B[0] + (double)my * G.B[1] + (double)mz * G.B[2]);
    gx += (T)(-G.V * G.Ms0 * G.B[0]);
    gy += (T)(-G.V * G.Ms0 * G.B[1]);
    gz += (T)(-G.V * G.Ms0 * G.B[2]);
    const double dq = l2 - G.me2;
    acc[5] += G.c2 * l2 + G.c4 * dq * dq;
    const T lc = (T)(2.0 * G.c2) + (T)(4.0 * G.c4) * (l2t - (T)G.me2);
    gx += lc * mx;
    gy += lc * my;
    gz += lc * mz;
    if (Hd) {
      const double hx = Hd[3 * q], hy = Hd[3 * q + 1], hz = Hd[3 * q + 2];
      acc[6] += -0.5 * mu0 * G.V * G.Ms0 * ((double)mx * hx + (double)my * hy + (double)mz * hz);
      const T f = (T)(-mu0 * G.V * G.Ms0);
      gx += f * (T)hx;
      gy += f * (T)hy;
      gz += f * (T)hz;
    }
    if (dEdm) {
      dEdm[3 * q] = gx;
      dEdm[3 * q + 1] = gy;
      dEdm[3 * q + 2] = gz;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    double v = acc[kk];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][kk] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double s = 0;
    for (int w = 0; w < kReduceBlock / 32; ++w) s += red[w][threadIdx.x];
    part[8LL * blockIdx.x + threadIdx.x] = s;
  }
}

__global__ void k_grad_final(const double *part, int nblocks, double *out8) {
  __shared__ double red[8][32];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 8; ++k) acc[k] += part[8LL * b + k];
  for (int k = 0; k < 8; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    out8[threadIdx.x] = s;
  }
}

void launch_energy_grad(const Launch &L, const ChainDev *chains_d, int c, long long ncell, const void *m,
                        bool fp64, const double *Hd, const GradCoef &G, void *dEdm, double *part,
                        double *out8) {
  const int nb = (int)((ncell + kReduceBlock * 4 - 1) / (kReduceBlock * 4));
  if (fp64)
    k_energy_grad<double><<<nb, kReduceBlock, 0, L.stream>>>(chains_d, c, (const double *)m, Hd, G,
                                                              (double *)dEdm, part);
  else
    k_energy_grad<float><<<nb, kReduceBlock, 0, L.stream>>>(chains_d, c, (const float *)m, Hd, G,
                                                             (float *)dEdm, part);
  k_grad_final<<<1, 256, 0, L.stream>>>(part, nb, out8);
  *L.counter += 2;
}

}  // namespace mmc
