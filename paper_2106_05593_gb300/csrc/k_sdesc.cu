// Zero-temperature steepest descent (the paper's SDesc comparison method,
// Sec. III) on one chain, FP64.  Directions u_i = m_i / m_e with |m_i| held at
// m_e(T): the tangential gradient g_i = m_e (G_i - (G_i . u_i) u_i) of the
// energy gradient G = dE/dm (k_grad.cu), a step u_i <- normalize(u_i - tau g_i)
// with Barzilai-Borwein step sizes chosen on the host from the block sums this
// file reduces (s.s, s.y, y.y with s = u - u_prev, y = g - g_prev, the largest
// |g_i|^2 and the largest normalized torque |u_i x h_i| / |h_i|).
#include "mmc_internal.h"

namespace mmc {

constexpr int kSdBlock = 256;

// state of the chain (split float4) -> unit directions u (natural order) and m = me u
__global__ void k_sd_init(const ChainDev *chains, int c, const float4 *mstate, double me, double *u, double *m) {
  const ChainDev &ch = chains[c];
  const long long n = ch.ncell;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % ch.nx);
    const int row = (int)(q / ch.nx);
    const int j = row % ch.ny, k = row / ch.ny;
    const int col = (i + j + k) & 1;
    const long long si = (long long)col * ch.nrows * ch.hx + (long long)row * ch.hx + (i >> 1);
    const float4 v = mstate[ch.m_off + si];
    double x = v.x, y = v.y, z = v.z;
    const double l = sqrt(x * x + y * y + z * z);
    if (l > 0) { x /= l; y /= l; z /= l; } else { x = 1; y = 0; z = 0; }
    u[3 * q] = x; u[3 * q + 1] = y; u[3 * q + 2] = z;
    m[3 * q] = me * x; m[3 * q + 1] = me * y; m[3 * q + 2] = me * z;
  }
}

// tangential gradient and the block sums [ss, sy, yy, max |g|^2, max torque]
__global__ void __launch_bounds__(kSdBlock) k_sd_dir(long long n, double me, const double *u, const double *G,
                                                     double *g, const double *up, const double *gp, double *part) {
  double ss = 0, sy = 0, yy = 0, gmax = 0, tmax = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double u0 = u[3 * q], u1 = u[3 * q + 1], u2 = u[3 * q + 2];
    const double G0 = G[3 * q], G1 = G[3 * q + 1], G2 = G[3 * q + 2];
    const double d = G0 * u0 + G1 * u1 + G2 * u2;
    const double g0 = me * (G0 - d * u0), g1 = me * (G1 - d * u1), g2 = me * (G2 - d * u2);
    g[3 * q] = g0; g[3 * q + 1] = g1; g[3 * q + 2] = g2;
    const double s0 = u0 - up[3 * q], s1 = u1 - up[3 * q + 1], s2 = u2 - up[3 * q + 2];
    const double y0 = g0 - gp[3 * q], y1 = g1 - gp[3 * q + 1], y2 = g2 - gp[3 * q + 2];
    ss += s0 * s0 + s1 * s1 + s2 * s2;
    sy += s0 * y0 + s1 * y1 + s2 * y2;
    yy += y0 * y0 + y1 * y1 + y2 * y2;
    const double gn2 = g0 * g0 + g1 * g1 + g2 * g2;
    const double Gn2 = me * me * (G0 * G0 + G1 * G1 + G2 * G2);
    gmax = fmax(gmax, gn2);
    tmax = fmax(tmax, Gn2 > 0 ? sqrt(gn2 / Gn2) : 0.0);
  }
  __shared__ double red[5][kSdBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_down_sync(0xffffffffu, ss, o);
    sy += __shfl_down_sync(0xffffffffu, sy, o);
    yy += __shfl_down_sync(0xffffffffu, yy, o);
    gmax = fmax(gmax, __shfl_down_sync(0xffffffffu, gmax, o));
    tmax = fmax(tmax, __shfl_down_sync(0xffffffffu, tmax, o));
  }
  if (lane == 0) { red[0][w] = ss; red[1][w] = sy; red[2][w] = yy; red[3][w] = gmax; red[4][w] = tmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kSdBlock / 32; ++k) {
      red[0][0] += red[0][k]; red[1][0] += red[1][k]; red[2][0] += red[2][k];
      red[3][0] = fmax(red[3][0], red[3][k]); red[4][0] = fmax(red[4][0], red[4][k]);
    }
    for (int k = 0; k < 5; ++k) part[5 * blockIdx.x + k] = red[k][0];
  }
}

// fixed-order final reduction of the block sums (deterministic)
__global__ void k_sd_final(const double *part, int nblocks, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b) {
    r[0] += part[5 * b]; r[1] += part[5 * b + 1]; r[2] += part[5 * b + 2];
    r[3] = fmax(r[3], part[5 * b + 3]); r[4] = fmax(r[4], part[5 * b + 4]);
  }
  for (int k = 0; k < 5; ++k) out[k] = r[k];
}

// u_prev <- u, g_prev <- g, u <- normalize(u - tau g), m <- me u
__global__ void k_sd_step(long long n, double me, double tau, double *u, const double *g, double *up, double *gp,
                          double *m) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    double v[3];
    double l2 = 0;
    for (int a = 0; a < 3; ++a) {
      up[3 * q + a] = u[3 * q + a];
      gp[3 * q + a] = g[3 * q + a];
      v[a] = u[3 * q + a] - tau * g[3 * q + a];
      l2 += v[a] * v[a];
    }
    const double il = 1.0 / sqrt(l2);
    for (int a = 0; a < 3; ++a) {
      u[3 * q + a] = v[a] * il;
      m[3 * q + a] = me * v[a] * il;
    }
  }
}

// natural-order m back into the chain's split float4 state (grain ids kept)
__global__ void k_sd_store(const ChainDev *chains, int c, const double *m, float4 *mstate) {
  const ChainDev &ch = chains[c];
  const long long n = ch.ncell;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % ch.nx);
    const int row = (int)(q / ch.nx);
    const int j = row % ch.ny, k = row / ch.ny;
    const int col = (i + j + k) & 1;
    const long long si = (long long)col * ch.nrows * ch.hx + (long long)row * ch.hx + (i >> 1);
    float4 v = mstate[ch.m_off + si];
    v.x = (float)m[3 * q]; v.y = (float)m[3 * q + 1]; v.z = (float)m[3 * q + 2];
    mstate[ch.m_off + si] = v;
  }
}

static int sd_grid(long long n) {
  long long b = (n + kSdBlock - 1) / kSdBlock;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

int sd_blocks(long long n) { return sd_grid(n); }

void launch_sd_init(const Launch &L, const ChainDev *chains, int c, long long n, const float4 *mstate, double me,
                    double *u, double *m) {
  k_sd_init<<<sd_grid(n), kSdBlock, 0, L.stream>>>(chains, c, mstate, me, u, m);
  ++*L.counter;
}

void launch_sd_dir(const Launch &L, long long n, double me, const double *u, const double *G, double *g,
                   const double *up, const double *gp, double *part, double *out5) {
  const int nb = sd_grid(n);
  k_sd_dir<<<nb, kSdBlock, 0, L.stream>>>(n, me, u, G, g, up, gp, part);
  k_sd_final<<<1, 32, 0, L.stream>>>(part, nb, out5);
  *L.counter += 2;
}

void launch_sd_step(const Launch &L, long long n, double me, double tau, double *u, const double *g, double *up,
                    double *gp, double *m) {
  k_sd_step<<<sd_grid(n), kSdBlock, 0, L.stream>>>(n, me, tau, u, g, up, gp, m);
  ++*L.counter;
}

void launch_sd_store(const Launch &L, const ChainDev *chains, int c, long long n, const double *m, float4 *mstate) {
  k_sd_store<<<sd_grid(n), kSdBlock, 0, L.stream>>>(chains, c, m, mstate);
  ++*L.counter;
}

}  // namespace mmc
