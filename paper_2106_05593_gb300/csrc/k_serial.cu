// Serial form of the MMC iteration (App. B): the cells of a chain are visited
// one at a time in index order i + nx (j + ny k), and after every accepted move
// the demag field of the whole chain is updated by -N(r - q) . dM_q, so that
// every move's Eq. 14 term sees the field of the current state.  Optionally the
// self term (mu0 V / 2) Ms0^2 dm . N(0) . dm is added, which makes each move's
// demag energy change exact.
//
// One thread block per chain.  The block first draws every cell's proposal in
// parallel (a cell's proposal depends only on its own moment and its Philox
// numbers, both fixed until the cell is visited) together with the cell-local
// part of the decision (longitudinal, anisotropy, the optional demag self term,
// the length factor and ln u3).  Then one thread walks the cells in order, adding the
// neighbour terms (exchange, DMI) and the field term against the current
// moments and field, while after each accepted move all threads of the block
// update the field of every cell from the real-space Newell tensor.  When the
// moments, the field and the tensor fit, they live in shared memory.
#include "mmc_internal.h"
#include "philox.cuh"
#include "trial.cuh"

namespace mmc {

struct SerialArgs {
  const ChainDev *chains;
  ChainState *st;
  float4 *m;
  float4 *heff;                 // h = zee (B + mu0 H_d), split layout; refreshed before every sweep
  const float4 *tab;
  const float *ms;
  const float *const *oct;      // per tensor set: [6][oz][oy][ox] real-space tensor, offsets >= 0
  const int4 *oct_dim;          // per tensor set: (ox, oy, oz, 0)
  float4 *prop;                 // proposals (m', local decision part), split layout like m
  const unsigned *sweep_base;
  unsigned sweep_off;
  unsigned key0, key1;
  int self;                     // add the demag self term
  size_t smem_limit;            // shared memory available to a block
};

constexpr int kSerialThreads = 1024;   // 32 x 32: x over i, y over rows

// shared-memory bytes of a chain: m and h (2 S float4 each) and the compact
// tensor (ncomp x nx ny nz floats)
__host__ __device__ inline size_t serial_smem_bytes(const ChainDev &ch) {
  const size_t slots = 2 * (size_t)ch.nrows * ch.hx;
  const int ncomp = ch.nz > 1 ? 6 : 4;
  return 2 * slots * sizeof(float4) + (size_t)ncomp * ch.ncell * sizeof(float);
}

template <bool PERCELL>
__global__ void __launch_bounds__(kSerialThreads, 1) k_serial_sweep(SerialArgs A) {
  extern __shared__ float4 sm4[];
  const int c = blockIdx.x;
  const ChainDev &ch = A.chains[c];
  const int nx = ch.nx, ny = ch.ny, nz = ch.nz, hx = ch.hx, nrows = ch.nrows;
  const long long S = (long long)nrows * hx;
  const int flags = ch.flags;
  const bool demag = (flags & F_DEMAG) != 0;
  const int ncomp = nz > 1 ? 6 : 4;
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const bool use_smem = serial_smem_bytes(ch) <= A.smem_limit;

  // state: moments, field and tensor in shared memory when they fit
  float4 *mg = A.m + ch.m_off;
  float4 *hg = demag ? A.heff + ch.h_off : nullptr;
  float4 *mm = mg, *hh = hg;
  const float *tn = nullptr;
  long long tstride = 0;        // component stride of the tensor
  int tsx = 1, tsy = 1;         // x and y strides of the tensor
  if (demag) {
    const int4 od = A.oct_dim[ch.spec];
    tn = A.oct[ch.spec];
    tstride = (long long)od.x * od.y * od.z;
    tsx = od.x;
    tsy = od.y;
  }
  if (use_smem) {
    mm = sm4;
    hh = sm4 + 2 * S;
    for (long long t = tid; t < 2 * S; t += kSerialThreads) {
      mm[t] = mg[t];
      if (demag) hh[t] = hg[t];
    }
    if (demag) {
      float *ts = reinterpret_cast<float *>(sm4 + 4 * S);
      const long long nc = ch.ncell;
      for (long long t = tid; t < nc; t += kSerialThreads) {
        const int x = (int)(t % nx), y = (int)((t / nx) % ny), z = (int)(t / ((long long)nx * ny));
        const long long src = ((long long)z * tsy + y) * tsx + x;
        for (int q = 0; q < ncomp; ++q) ts[q * nc + t] = tn[q * tstride + src];
      }
      tn = ts;
      tstride = nc;
      tsx = nx;
      tsy = ny;
    }
  }
  const unsigned sweep = *A.sweep_base + A.sweep_off;
  const float omc = A.st[c].omc;
  float4 *pr = A.prop + ch.m_off;
  __syncthreads();

  // 1. proposals and the cell-local part of every decision (parallel)
  for (long long t = tid; t < 2 * S; t += kSerialThreads) {
    const int color = t >= S ? 1 : 0;
    const long long q = t - color * S;
    const int row = (int)(q / hx), s = (int)(q - (long long)row * hx);
    const int k = row / ny, j = row - k * ny;
    const int i = 2 * s + ((j + k + color) & 1);
    if (i >= nx) continue;
    const float4 a = mm[t];
    const CellMat M = cell_material<PERCELL>(ch, A.tab, S, t);
    const unsigned cell = (unsigned)i + (unsigned)nx * (unsigned)row;
    const uint4 r = philox4x32_10(make_uint4(cell, sweep, (unsigned)ch.chain, 0u), make_uint2(A.key0, A.key1));
    const float u0 = uniform01(r.x), u1 = uniform01(r.y), u2 = uniform01(r.z), u3 = uniform01(r.w);
    Move v = move_length(a, M.me2h, M.me2l);
    move_direction(v, a, M.sigma, omc, u0, u1, u2);
    float loc = longitudinal_change(v, M.p2, M.p4) + anisotropy_change(v, flags, M.k1, M.k2, M.ex, M.ey, M.ez);
    if (demag && A.self) {
      // self term (mu0 V / 2) Ms0^2 dm . N(0) . dm in kT: (mu0 / 2) zee Ms0 (...)
      const float Ms = ch.ms_off >= 0 ? A.ms[ch.ms_off + t] : ch.Ms0;
      const float ns = v.dmx * v.dmx * tn[0] + v.dmy * v.dmy * tn[tstride] + v.dmz * v.dmz * tn[2 * tstride];
      loc += 0.5f * (float)mu0 * M.zee * Ms * ns;
    }
    loc = loc - 4.f * log1p_move(v.tt) + __logf(u3);
    pr[t] = make_float4(v.mpx, v.mpy, v.mpz, loc);
  }
  __syncthreads();

  // 2. the walk in index order
  __shared__ float bc[4];       // broadcast: accepted, mu0 Ms0 dm
  unsigned long long nacc = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j) {
      const int row = j + ny * k;
      for (int i = 0; i < nx; ++i) {
        const int color = (i + j + k) & 1;
        const long long idx = (long long)color * S + (long long)row * hx + (i >> 1);
        if (tid == 0) {
          const float4 a = mm[idx];
          const float4 P = pr[idx];
          float4 nb[6];
          float w[6];
          load_neighbours(ch.pbc, (flags & F_GRAIN) != 0, ch.gscale, nx, ny, nz, hx, mm + (long long)(1 - color) * S, a,
                          i, j, k, row, i >> 1, i & 1, nb, w);
          float bs = 1.f, zee = ch.zee;
          if (PERCELL) {
            const float4 t1 = A.tab[ch.t_off + 2 * S + idx];
            zee = t1.x;
            bs = t1.w;
          }
          float hxs, hys, hzs;
          if (demag) {
            const float4 h = hh[idx];
            hxs = h.x; hys = h.y; hzs = h.z;
          } else {
            hxs = zee * ch.Bx; hys = zee * ch.By; hzs = zee * ch.Bz;
          }
          Move v;
          v.mpx = P.x; v.mpy = P.y; v.mpz = P.z;
          v.dmx = P.x - a.x; v.dmy = P.y - a.y; v.dmz = P.z - a.z;
          const float fex = exchange_change(v, a, nb, w, ch.wx * bs, ch.wy * bs, ch.wz * bs, nz > 1);
          const float flin = linear_change(v, nb, w, ch.cdx * bs, ch.cdy * bs, (flags & F_DMI) != 0, hxs, hys, hzs);
          const bool acc = (fex + flin) + P.w < 0.f;
          if (acc) {
            mm[idx] = make_float4(P.x, P.y, P.z, a.w);
            ++nacc;
            const float Ms = ch.ms_off >= 0 ? A.ms[ch.ms_off + idx] : ch.Ms0;
            const float g = (float)mu0 * Ms;
            bc[1] = g * v.dmx; bc[2] = g * v.dmy; bc[3] = g * v.dmz;
          }
          bc[0] = acc ? 1.f : 0.f;
        }
        if (!demag) continue;   // nothing to share: thread 0 walks alone
        __syncthreads();
        if (bc[0] != 0.f) {
          // h_r -= zee_r mu0 N(r - q) . (Ms0_q dm_q) for every cell r of the chain
          const float gx = bc[1], gy = bc[2], gz = bc[3];
          for (int r2 = threadIdx.y; r2 < nrows; r2 += 32) {
            const int kr = r2 / ny, jr = r2 - kr * ny;
            const int dy = jr - j, dz = kr - k;
            const int ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
            const float sy = dy < 0 ? -1.f : 1.f, sz = dz < 0 ? -1.f : 1.f;
            const long long tb = ((long long)az * tsy + ay) * tsx;
            for (int ir = threadIdx.x; ir < nx; ir += 32) {
              const int dx = ir - i;
              const int ax = dx < 0 ? -dx : dx;
              const float sx = dx < 0 ? -1.f : 1.f;
              const long long to = tb + ax;
              const float Nxx = tn[to], Nyy = tn[tstride + to], Nzz = tn[2 * tstride + to];
              const float Nxy = sx * sy * tn[3 * tstride + to];
              float Nxz = 0.f, Nyz = 0.f;
              if (ncomp == 6) {
                Nxz = sx * sz * tn[4 * tstride + to];
                Nyz = sy * sz * tn[5 * tstride + to];
              }
              const int cr = (ir + jr + kr) & 1;
              const long long ri = (long long)cr * S + (long long)r2 * hx + (ir >> 1);
              const float zr = PERCELL ? A.tab[ch.t_off + 2 * S + ri].x : ch.zee;
              float4 h = hh[ri];
              h.x -= zr * (Nxx * gx + Nxy * gy + Nxz * gz);
              h.y -= zr * (Nxy * gx + Nyy * gy + Nyz * gz);
              h.z -= zr * (Nxz * gx + Nyz * gy + Nzz * gz);
              hh[ri] = h;
            }
          }
        }
        __syncthreads();
      }
    }
  __syncthreads();

  if (use_smem)
    for (long long t = tid; t < 2 * S; t += kSerialThreads) mg[t] = mm[t];
  if (tid == 0) {
    atomicAdd(&A.st[c].win_acc, nacc);
    atomicAdd(&A.st[c].win_att, (unsigned long long)ch.ncell);
  }
}

void launch_serial_sweep(const Launch &L, const SerialLaunch &P) {
  SerialArgs A;
  A.chains = P.chains; A.st = P.st; A.m = P.m; A.heff = P.heff; A.tab = P.tab; A.ms = P.ms;
  A.oct = P.oct; A.oct_dim = P.oct_dim; A.prop = P.prop; A.sweep_base = P.sweep_base;
  A.sweep_off = P.sweep_off; A.key0 = P.key0; A.key1 = P.key1; A.self = P.self ? 1 : 0;
  A.smem_limit = P.smem;
  const dim3 blk(32, 32);
  if (P.percell) k_serial_sweep<true><<<P.nchains, blk, P.smem, L.stream>>>(A);
  else k_serial_sweep<false><<<P.nchains, blk, P.smem, L.stream>>>(A);
  ++*L.counter;
}

size_t serial_smem_need(const ChainDev &ch) { return serial_smem_bytes(ch); }

cudaError_t serial_set_smem_limit(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_serial_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_serial_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace mmc
