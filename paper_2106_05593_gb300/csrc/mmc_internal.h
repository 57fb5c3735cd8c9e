// Internal declarations shared by the library's translation units.
// Not part of the C ABI (include/mmc.h is).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "checked.cuh"

namespace mmc {

// Programmatic dependent launch.  The sublattice-pass, window-step and
// observables kernels are launched with launch_pdl, so such a kernel may be
// scheduled while the previous kernel of its stream drains; each of them first
// waits for the previous grid to complete and its memory to be visible
// (griddepcontrol.wait), then lets its own successor be scheduled (the
// successor waits the same way before it touches memory).  Small, launch-bound
// batches gain from it; the demag kernels, whose blocks hold large shared-memory
// tiles, are launched plainly (scheduled early, they slowed single-chain runs).
__device__ __forceinline__ void pdl_enter() {
#if defined(__CUDA_ARCH__)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace mmc

namespace mmc {

// CODATA 2018 SI values
constexpr double kB = 1.380649e-23;
constexpr double muB = 9.2740100783e-24;
constexpr double mu0 = 1.25663706212e-6;
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxFFT = 4096;        // largest padded FFT length per axis (twiddle table length)
constexpr int kMaxDemagImages = 64;  // largest number of periodic demag images per side
constexpr int kHistMax = 1024;       // largest histogram bin count
constexpr int kSweepBlock = 256;     // threads per sweep-pass block
constexpr int kReduceBlock = 256;

// chain flag bits
enum : int {
  F_GRAIN = 2,     // grain ids in m.w, bonds between grains scaled
  F_DMI = 4,
  F_ANIS = 8,      // uniaxial anisotropy present
  F_CUBIC = 16,    // cubic anisotropy
  F_DEMAG = 32,    // h_eff array present (demag on)
};

// Per-chain constants, device resident.  Energies are in units of kT (of the
// chain temperature, or of a reference T_ref for per-cell chains, whose table
// carries bscale = T_ref / T_cell for the bond weights).
struct __align__(16) ChainDev {
  // the sweep kernel reads the first 128 bytes as eight 16-byte vectors
  int nx, ny, nz;
  int hx;             // sublattice slots per row: (nx + 1) / 2
  int nrows;          // ny * nz
  int pbc;            // bit a: axis a periodic
  int flags;
  int chain;          // chain index (Philox counter word 2)
  unsigned hx_m, ny_m, nx_m;   // division by hx, ny and nx: multiply-shift constants
  int spec;           // tensor-spectrum set index
  int hx_l, ny_l, nx_l;        // (Granlund & Montgomery's round-up method, l = ceil(log2 d))
  float gscale;       // bond scale across grains
  float wx, wy, wz;   // exchange bond weights V A0 / (h^2 kT)
  float cdx;          // DMI weights V D0 / (h kT), x bonds
  float cdy;          // y bonds
  float p2, p4;       // longitudinal: dF/kT = dq (p2 + p4 (2 (|m|^2 - me2) + dq))
  float me2h;         // m_e^2 as a float-float pair (0 at and above Tc)
  float me2l;
  float sigma;        // length-move width (Eq. 13, capped)
  float zee;          // V Ms0 / kT  (1/T)
  float k1, k2;       // V K1(T) / kT, V K2(T) / kT
  float ex, ey, ez;   // easy axis
  float Bx, By, Bz;   // applied field (T)
  float Ms0;          // A/m (uniform chains)
  long long m_off;    // float4 index of the red array in the m arena; black follows
  long long h_off;    // float4 index of the red h_eff array (split layout), or -1
  long long t_off;    // float4 index of the per-cell table (3 x 2 x nrows*hx float4), or -1
  long long ms_off;   // float index of per-cell Ms0 (split layout), or -1
  long long ncell;
  long long s_off;    // complex element index of the spectrum buffer
  int Px, Py, Pz;     // padded FFT sizes
  int Sx;             // row stride (complex elements) of the spectrum buffer
  int lx, ly, lz;     // log2 of the padded sizes
  int circ;           // bit a: axis a periodic for demag with P_a = n_a (circular transform, no padding)
  double Ms0d;        // Ms0 in FP64 (convolution input of the FP64 path)
};

// Per-chain mutable state, device resident (plain data; part of checkpoints).
struct ChainState {
  unsigned long long win_acc;    // accepted moves in the current window
  unsigned long long win_att;    // attempted moves in the current window
  unsigned long long last_acc;   // of the last completed window
  unsigned long long last_att;
  float theta_deg;
  float omc;                     // 1 - cos(theta)
  double sum_m[3];               // snapshot accumulators
  double sum_len, sum_len2;
  unsigned long long nsamples;
  unsigned long long nsnap;
  unsigned long long nonfinite;
};

// FP64 energy coefficients of a uniform chain (J), see k_reduce.cu
struct EnergyCoef {
  double cex[3];      // V A0 / h_a^2
  double cdmi[2];     // V D0 / h_a
  double c2, c4, me2; // F_l = c2 m^2 + c4 (m^2 - me2)^2
  double Ms0, K1T, K2T, e[3];
  double B[3];
  double V;
  int cubic;
};

// coefficients of the differentiable energy (J), see k_grad.cu
struct GradCoef {
  double cex[3];      // V A0 / h_a^2
  double cdmi[2];     // V D0 / h_a
  double vh2[3];      // V / h_a^2   (dE/dA0 per unit bond sum)
  double vh[2];       // V / h_a     (dE/dD0)
  double c2, c4, me2; // F_l = c2 m^2 + c4 (m^2 - me2)^2
  double Ms0, K1T, K2T, Kscale, e[3];
  double B[3];
  double V;
  int cubic, anis, dmi;
};

// q / d for 32-bit unsigned q with precomputed (m, l) of d (l = 0 means d = 1)
__host__ __device__ inline void divmagic(unsigned d, unsigned &m, int &l) {
  if (d <= 1) { m = 0; l = 0; return; }
  l = 0;
  while ((1u << l) < d && l < 31) ++l;
  if ((1ull << l) < d) l = 32;
  m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
}
#ifdef __CUDACC__
__device__ __forceinline__ unsigned divq(unsigned q, unsigned m, int l) {
  if (l == 0) return q;
  const unsigned t = __umulhi(m, q);
  return (t + ((q - t) >> 1)) >> (l - 1);
}
#endif

// message returned by mmc_last_error() on the calling thread
void set_last_error(const char *msg);

// ---------------------------------------------------------------------------
// host-side physics (host_physics.cpp)
double langevin(double x);
double langevin_deriv(double x);
double me_of_T(double T, double Tc);
double chi_of_T(double T, double Tc, double mu);
double sigma_of_T(double T, double Tc, double mu, double V, double Ms0, double cap);
void long_coeffs(double T, double Tc, double mu, double V, double Ms0, double *c2, double *c4);
double rms_len_eq7(double T, double Tc, double mu, double V, double Ms0);
void demag_tensor(const double h[3], const double R[3], double out[6]);
// Periodic demag along the axes a with per[a] set (extent n[a]): the kernel is the
// tensor summed over `images` periodic images on each side, each offset at its
// minimal image, the half period split between its two minimal images.  With
// images == 0 (or no periodic axis) the convolution has open boundaries.  The
// zero-padded convolution with this kernel on offsets -(n-1)..n-1 is the
// circular convolution exactly.
// A periodic axis whose extent is a power of two (>= kCircMin) is transformed
// circularly (circ[a]: transform length n_a, no zero padding); the kernel's
// half-period offset then reaches mesh cells and is kept in the spectrum.
struct DemagPeriodic {
  int n[3] = {1, 1, 1};
  int per[3] = {0, 0, 0};
  int circ[3] = {0, 0, 0};
  int images = 0;
  bool any() const { return images > 0 && (per[0] || per[1] || per[2]); }
  bool operator==(const DemagPeriodic &o) const {
    if (any() != o.any()) return false;
    if (!any()) return true;
    for (int a = 0; a < 3; ++a)
      if (per[a] != o.per[a] || circ[a] != o.circ[a] || (per[a] && n[a] != o.n[a])) return false;
    return images == o.images;
  }
};
constexpr int kCircMin = 8;          // smallest periodic extent transformed circularly
void demag_spectra(const double h[3], int Px, int Py, int Pz, std::vector<double> &out,
                   const DemagPeriodic &pd = DemagPeriodic());
void demag_octant(const double h[3], int ox, int oy, int oz, std::vector<double> &oct,
                  const DemagPeriodic &pd = DemagPeriodic());

// ---------------------------------------------------------------------------
// launches
struct Launch {
  cudaStream_t stream;
  long long *counter;   // kernel launch counter
};

struct SweepLaunch {
  const ChainDev *chains;
  ChainState *st;
  const int2 *blk_desc;         // per block: (chain, block index within the chain)
  int blk_base;                 // first block of this launch in the block tables
  int nblocks;
  float4 *m;
  const float4 *heff;
  const float4 *tab;
  const unsigned *sweep_base;
  unsigned sweep_off;
  unsigned key0, key1;
  int color;
  bool percell;
  float omc_override;
  float *dec_dbg;
  signed char *acc_dbg;
  int nstripes, stripe;         // nstripes > 1: only the band `stripe` of rows of every chain
  bool flat;                    // every chain has nz == 1
  // banded pass with shared-memory halo tiles (uniform one-cell-thick batches)
  bool band;
  const int4 *items;            // per band: (chain, first row, rows, 0), by chain
  int i0, i1;                   // items of this launch
  int band_grid;                // resident blocks (SMs x blocks per SM)
  int stage_own, stage_other;   // float4 capacity of a stage's own-colour and other-colour tiles
  unsigned max_polls;           // bound of a wait for a band's copies
  int *err;                     // device error word
  int wait_test;                // test hook (mmc_options.wait_test)
  MmcCheck *ck;                 // checked builds: the record (checked.cuh)
  int blk_total, nchains, nitems;   // sizes of the block table, chain table and item table
};
constexpr int MMC_ERR_TIMEOUT_CODE = -3;   // mmc_status MMC_ERR_TIMEOUT
void launch_sweep_pass(const Launch &L, const SweepLaunch &P);
size_t band_smem_bytes(int stage_own, int stage_other);
cudaError_t band_set_smem(size_t bytes);
int band_blocks_per_sm(size_t bytes);
void launch_advance(const Launch &L, ChainState *st, int nchains, unsigned by, unsigned *sweep_base,
                    int adapt_now, int adapt, float tmin, float tmax);

// serial exact-demag sweep (k_serial.cu)
struct SerialLaunch {
  const ChainDev *chains;
  ChainState *st;
  float4 *m;
  float4 *heff;
  const float4 *tab;
  const float *ms;
  const float *const *oct;      // per tensor set: real-space tensor [6][oz][oy][ox]
  const int4 *oct_dim;
  float4 *prop;                 // scratch with the layout of m
  const unsigned *sweep_base;
  unsigned sweep_off;
  unsigned key0, key1;
  int nchains;
  bool percell;
  bool self;                    // add the demag self term to every move
  size_t smem;                  // dynamic shared memory per block (chains needing more run from global memory)
};
void launch_serial_sweep(const Launch &L, const SerialLaunch &P);
size_t serial_smem_need(const ChainDev &ch);
cudaError_t serial_set_smem_limit(size_t bytes);

// steepest-descent minimizer (k_sdesc.cu)
int sd_blocks(long long n);
void launch_sd_init(const Launch &L, const ChainDev *chains, int c, long long n, const float4 *mstate, double me,
                    double *u, double *m);
void launch_sd_dir(const Launch &L, long long n, double me, const double *u, const double *G, double *g,
                   const double *up, const double *gp, double *part, double *out5);
void launch_sd_step(const Launch &L, long long n, double me, double tau, double *u, const double *g, double *up,
                    double *gp, double *m);
void launch_sd_store(const Launch &L, const ChainDev *chains, int c, long long n, const double *m, float4 *mstate);

struct DemagLaunch {
  const ChainDev *chains;
  const float4 *m;
  const float4 *tab;
  const float *ms;
  const float *ms_lo;           // per-cell Ms0 minus its FP32 value (or null)
  void *spec;
  const void *const *nhat;
  const void *twiddle;
  float4 *heff;
  double *Hd;
  int Hd_chain;
  const int *rows_chain;
  const long long *rows_first;
  int rows_blocks, rows_threads;
  size_t rows_smem;
  const int *cols_chain;
  const long long *cols_first;
  int cols_blocks, cols_threads, cols_per_block;
  size_t cols_smem;
  cudaEvent_t *ev;              // optional: 4 events recorded around the three kernels
  const void *m_nat;            // optional natural-order m (float or double, as the plan)
  double Ms_override;           // uniform Ms0 used with m_nat
  bool il2d;                    // 2D interleaved kernels (all chains Pz == 1)
  int fft_variant;              // FP32 2D kernels: 1 radix 16 (384 threads), 2 radix 32 (192 threads)
  size_t inv_smem;              // shared memory of the 2D inverse row kernel
  bool w32;                     // FP32 1024 x 1024 warp-transform kernels (k_demag_w32.cu)
  const void *const *nhatT;     // their tensor spectra, per set [comp][kx][kyq] (or null), kyq pitch kW32TensorPitch
  const void *tw1024;           // their 32 x 32 twiddle table
  const void *tmap_spec;        // their spectrum as a 2D tensor (CUtensorMap, host copy) for the column boxes
  int *err;                     // device error word of bounded waits
  MmcCheck *ck;                 // checked builds: the record (checked.cuh)
  int nchains;                  // entries of the chain table
  bool ff;                      // with fp64: float-float arithmetic in the generic kernels (nhat and
                                // twiddle tables in float-float, the spectrum as pairs of float pairs)
};
constexpr int kW32TensorPitch = 516;      // kyq = 0..512 padded to a 16-byte multiple of floats
constexpr int kW32Sx = 520;                // spectrum row stride of a 1024-point grid (513 kx, 32-byte multiple)
constexpr int kW32Tile = 4 * kW32Sx;       // complex values of one tile of four rows
void launch_w32(const Launch &L, const DemagLaunch &P);
void launch_w32_stage(const Launch &L, const DemagLaunch &P, int stage);   // 0 rows fwd, 1 cols, 2 rows inv
// the black pass fused with the forward row transforms (k_demag_w32.cu)
void launch_w32_black_rows_fwd(const Launch &L, const DemagLaunch &P, const SweepLaunch &Q);
// the inverse row transforms fused with the red pass (k_demag_w32.cu)
void launch_w32_rows_inv_red(const Launch &L, const DemagLaunch &P, const SweepLaunch &Q);
cudaError_t w32_set_smem();
// a chain the warp-transform path handles: one cell thick, padded grid 1024 x 1024, open demag
inline bool w32_chain(const ChainDev &D) {
  return D.nz == 1 && D.Pz == 1 && D.Px == 1024 && D.Py == 1024 && D.circ == 0 && D.Sx == 520;
}
// rows of a chain's spectrum buffer: 2D chains round up to tiles of four rows
inline long long spectrum_rows(const ChainDev &D) { return D.Pz == 1 ? ((D.nrows + 3) & ~3) : D.nrows; }
int il_elements(bool fp64);     // complex elements per block of the 2D kernels
int il_padded_elements(bool fp64);   // shared-memory elements those occupy (bank padding)
int il_padded_of(int e);             // shared-memory elements of e logical elements
int il_elements_small();             // block size of the 2-blocks-per-SM FP32 variant
void launch_demag(const Launch &L, const DemagLaunch &P, bool fp64);
cudaError_t demag_set_smem_limits();

// cuFFT comparison path (k_cufft.cu): chains of one padded size
struct CufftGroup {
  int Px = 1, Py = 1, Pz = 1;
  bool fp64 = false;
  int nchain = 0;
  int *chain_of = nullptr;     // device: chain index per slot
  void *real = nullptr;        // [slot][comp][Pz][Py][Px]
  void *cplx = nullptr;        // [slot][comp][Pz][Py][Px/2+1]
  int fwd = 0, inv = 0;        // cufftHandle
  bool planned = false;
};
cudaError_t make_cufft_plans(CufftGroup &G);
void destroy_cufft_plans(CufftGroup &G);
cudaError_t launch_cufft_group(const Launch &L, const CufftGroup &G, const ChainDev *chains_d,
                               const float4 *m, const float *ms, const float4 *tab, float4 *heff,
                               double *Hd, int Hd_slot, const void *const *nhat, cudaEvent_t *ev);

struct ObsLaunch {
  const ChainDev *chains;
  ChainState *st;
  const int *blk_chain;
  const long long *blk_first;   // nchains + 1 entries
  int nblocks, nchains;
  const float4 *m;
  double *part;
  unsigned long long *hist;
  int bins;
  float scale;
  double *out;
  int accumulate;
};
void launch_obs(const Launch &L, const ObsLaunch &P);

void launch_energy(const Launch &L, const ChainDev *chains_d, int c, long long slots,
                   const float4 *m, const double *etab, const double *Hd, const EnergyCoef &E,
                   double *part, double *out7);
void launch_energy_grad(const Launch &L, const ChainDev *chains_d, int c, long long ncell, const void *m,
                        bool fp64, const double *Hd, const GradCoef &G, void *dEdm, double *part,
                        double *out8);
void launch_check_finite(const Launch &L, const float4 *v, long long n, int *flag);
void launch_pack(const Launch &L, const ChainDev *chains_d, int c, long long slots, float4 *m,
                 const float4 *nat, int to_split);
void launch_init_random(const Launch &L, const ChainDev *chains_d, int c, long long slots, float4 *m,
                        unsigned key0, unsigned key1, const float *len_nat, float len);

}  // namespace mmc
