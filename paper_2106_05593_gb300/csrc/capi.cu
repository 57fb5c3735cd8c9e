// C ABI of the GB300 MMC library (include/mmc.h): context set-up, host tables,
// launch plans, the sweep loop (eager or CUDA-graph blocks of 100 iterations),
// measurements and checkpoints.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <filesystem>
#include <functional>
#include <fstream>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/mmc.h"
#include "mmc_internal.h"
#include "angles.h"
#include "terms.h"

using namespace mmc;

namespace {

thread_local std::string g_err;

mmc_status fail(mmc_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

// NVTX range for profilers (nsys, ncu --nvtx): every public call, and in eager
// execution every phase of an iteration; a no-op when no tool is attached
struct Trace {
  explicit Trace(const char *name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace &) = delete;
  Trace &operator=(const Trace &) = delete;
};

}  // namespace

void mmc::set_last_error(const char *msg) { g_err = msg; }

namespace {

#define CUDA_TRY(expr)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return fail(MMC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MMC_TRY(expr)                 \
  do {                                \
    mmc_status s_ = (expr);           \
    if (s_ != MMC_OK) return s_;      \
  } while (0)

// inside create: release the half-built context on failure
#define MMC_TRY_OR(expr)                          \
  do {                                            \
    mmc_status s_ = (expr);                       \
    if (s_ != MMC_OK) { mmc_destroy(c); return s_; } \
  } while (0)
#define CUDA_TRY_OR(expr)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      mmc_destroy(c);                                                                          \
      return fail(MMC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));           \
    }                                                                                          \
  } while (0)

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int pad_len(int n, bool axis_active) {
  if (!axis_active) return 1;
  int p = 2;
  while (p < 2 * n) p <<= 1;
  return p;
}

struct ChainHost {
  mmc_mesh mesh;
  double h[3];
  double V;
  double T, Tc, Ms0, K1, K2, mu;
  int cubic;
  bool percell;
  double Tref;
  long long ncell, slots;
  std::vector<double> me, chi, sigma;   // per cell (size 1 for uniform chains)
  EnergyCoef ecoef;
  std::vector<double> etab;             // per-cell energy table, 10 doubles per cell
  std::vector<float> init_len;          // per-cell initial length (natural order)
  std::vector<float> grain;             // natural order, or empty
  // temperature-independent inputs kept for mmc_set_temperature
  double e[3];                          // normalized easy axis
  int l1, l2;                           // exponents of m_e in K1(T), K2(T)
  std::vector<double> Ms0_cell, K1_cell, Tc_cell, eA_cell;   // copies of the per-cell inputs, or empty
};

// block tables of the 2D interleaved kernels for one block size E
struct IlTables {
  bool ok = false;
  int *rows_chain = nullptr, *cols_chain = nullptr;
  long long *rows_first = nullptr, *cols_first = nullptr;
  int rows_blocks = 0, cols_blocks = 0;
  size_t rows_smem = 0, cols_smem = 0, inv_smem = 0;
};

struct DemagPlan {
  IlTables small;                       // FP32 variant 3: E = 6144 (2 blocks per SM)
  IlTables w32;                         // FP32 variant 4: warp transforms, 1024 x 1024 grids only
  CUtensorMap tmap_spec;                // variant 4: the spectrum as a 2D tensor of tiles (column boxes)
  bool fp64 = false;
  bool ff = false;                      // fp64 plan run by the float-float generic kernels
  int nchain_table = 0;                 // entries of the chain table the plan indexes
  ChainDev *d_ch = nullptr;             // chain table the plan indexes
  int *rows_chain = nullptr;
  long long *rows_first = nullptr;
  int rows_blocks = 0, rows_threads = 0;
  size_t rows_smem = 0;
  int *cols_chain = nullptr;
  long long *cols_first = nullptr;
  int cols_blocks = 0, cols_threads = 0, cols_cc = 1;
  size_t cols_smem = 0;
  void *spec = nullptr;
  bool il2d = false;
  int fft_variant = 1;
  size_t inv_smem = 0;
  bool ready = false;
};

struct SpecSet {
  double h[3];
  int Px, Py, Pz;
  DemagPeriodic pd;                     // periodic axes of the convolution
  void *d32 = nullptr, *d64 = nullptr;
  void *d32t = nullptr;                 // FP32 [comp][kx][kyq] copy for the warp-transform path
};

struct GraphEntry {
  unsigned key0, key1;
  int sample_every;
  long long launches;
  cudaGraphExec_t exec;
};

}  // namespace

struct mmc_ctx {
  int nchains = 0;
  mmc_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool any_demag = false, any_percell = false;
  std::vector<ChainHost> hc;
  std::vector<ChainDev> ch;
  ChainDev *d_ch = nullptr;
  ChainState *d_st = nullptr, *d_st_dbg = nullptr;
  unsigned *d_sweep_base = nullptr, *d_dbg_sweep = nullptr;
  float4 *d_m = nullptr, *d_heff = nullptr, *d_tab = nullptr;
  float *d_ms = nullptr;
  float *d_ms_lo = nullptr;             // per-cell Ms0 minus its FP32 value (FP64 and float-float demag)
  long long m_total = 0, tab_total = 0, ms_total = 0;
  std::vector<SpecSet> specs;
  void **d_nhat32 = nullptr, **d_nhat64 = nullptr, **d_nhat32t = nullptr;
  void *d_tw32 = nullptr, *d_tw64 = nullptr, *d_tw1024 = nullptr;
  void **d_nhatff = nullptr;            // float-float tensor spectra (demag_fp64 = 2)
  void *d_twff = nullptr;               // float-float twiddle table
  int *d_sw_chain = nullptr;
  long long *d_sw_first = nullptr;
  int2 *d_sw_desc = nullptr;
  std::vector<long long> sw_first;
  int sw_blocks = 0;
  int *d_obs_chain = nullptr;
  long long *d_obs_first = nullptr;
  int obs_blocks = 0;
  double *d_part = nullptr;
  unsigned long long *d_hist_acc = nullptr, *d_hist_cur = nullptr;
  double *d_obs_out = nullptr;
  DemagPlan batch_plan;
  std::vector<CufftGroup> cf;           // cuFFT comparison path (demag_cufft)
  // chain groups whose iterations run concurrently on their own streams (the
  // tail of one group's kernels overlaps the other's); empty: one stream
  struct ChainGroup {
    int c0 = 0, c1 = 0;                 // chains [c0, c1)
    DemagPlan plan;                     // demag over the group (batch spectrum buffer)
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<ChainGroup> groups;
  cudaEvent_t ev_fork = nullptr;
  int tuned_variant = 0;                // FFT variant picked at create (0: not tuned)
  int tuned_groups = 0;                 // chain groups picked at create (0: not tuned)
  bool tune_cached = false;             // the picks came from the tuning cache
  double group_ms[3] = {0.0, 0.0, 0.0}; // per-iteration time with 1, 2, 3 groups when timed
  double tune_ms[4] = {0.0, 0.0, 0.0, 0.0};  // per-update time of the variants when tuned
  std::vector<DemagPlan> single[2];     // per chain and precision (0 FP32, 1 FP64), built lazily
  // serial exact-demag sweep: real-space tensors per set, proposals scratch
  bool serial_ready = false;
  float **d_oct = nullptr;
  int4 *d_oct_dim = nullptr;
  float4 *d_prop = nullptr;
  size_t serial_smem = 0;
  // steepest-descent minimizer scratch (sized for the largest chain, built lazily)
  double *d_sd = nullptr;       // u, m, u_prev, g_prev, G, g: 6 x 3 max_ncell
  double *d_sd_part = nullptr, *d_sd_out = nullptr;
  double *d_g8 = nullptr;
  double *d_Hd = nullptr, *d_eout = nullptr, *d_etab = nullptr;
  float4 *d_nat = nullptr;
  float4 *d_nat_all = nullptr;          // every chain in natural order (mmc_set_m_all / get_m_all)
  float *d_dec = nullptr;
  signed char *d_acc = nullptr;
  long long max_ncell = 0, max_slots = 0;
  bool all_flat = true;                 // every chain one cell thick (nz == 1)
  // banded sublattice pass with shared-memory halo tiles (k_sweep_band)
  bool band = false;
  int4 *d_items = nullptr;              // per band: (chain, first row, rows, 0), by chain
  std::vector<int> item_first;          // first item of every chain (nchains + 1 entries)
  int band_grid = 0, stage_own = 0, stage_other = 0;
  int *d_err = nullptr;                 // device error word of the kernels' bounded waits
  MmcCheck *d_check = nullptr;          // checked builds: the first out-of-range index (checked.cuh)
  long long launches = 0;
  uint64_t host_sweep = 0;
  bool heff_stale = true;               // state or field changed since the last demag update
  bool obs_fresh = false;               // current-state observables of all chains are up to date
  int *d_flag = nullptr;                // device scratch int (input checks)
  unsigned long long *d_ang = nullptr;  // angular histogram counters (kHistMax + 1)
  double *d_terms = nullptr;            // trial-term partials (blocks x 6) and sums (6)
  std::vector<GraphEntry> graphs;
  std::vector<void *> allocs;

  Launch L() { return Launch{stream, &launches}; }
};

namespace {

mmc_status dalloc(mmc_ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(MMC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return MMC_OK;
}

template <typename T>
mmc_status dalloc_t(mmc_ctx *c, T **p, size_t count) {
  void *v = nullptr;
  mmc_status s = dalloc(c, &v, count * sizeof(T));
  *p = static_cast<T *>(v);
  return s;
}

template <typename T>
mmc_status upload(mmc_ctx *c, T **p, const std::vector<T> &v) {
  MMC_TRY(dalloc_t(c, p, std::max<size_t>(v.size(), 1)));
  if (!v.empty()) CUDA_TRY(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return MMC_OK;
}

// thermodynamic state of one (T, Tc) pair, Eqs. 7-9 and 13
struct Thermo {
  double me, chi, sigma, c2, c4, me2;   // F_l = c2 m^2 + c4 (m^2 - me2)^2
};

Thermo thermo(double T, double Tc, double mu, double V, double Ms0, double cap) {
  Thermo t;
  t.me = me_of_T(T, Tc);
  t.chi = chi_of_T(T, Tc, mu);
  t.sigma = sigma_of_T(T, Tc, mu, V, Ms0, cap);
  double c2, c4;
  long_coeffs(T, Tc, mu, V, Ms0, &c2, &c4);
  const double Tg = std::fabs(T - Tc) < 1e-3 ? (T < Tc ? Tc - 1e-3 : Tc + 1e-3) : T;
  if (Tg < Tc) {
    t.c2 = 0.0; t.c4 = c4; t.me2 = t.me * t.me;
  } else {
    t.c2 = c2; t.c4 = c4; t.me2 = 0.0;
  }
  return t;
}

void split_f(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

template <typename F>
void parallel_for(long long n, F fn) {
  const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < 4096 || nth == 1) {
    for (long long i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back([&, t]() {
      for (long long i = t; i < n; i += nth) fn(i);
    });
  for (auto &x : th) x.join();
}

bool has_percell(const mmc_chain_desc &d) {
  const mmc_material &mt = d.material;
  return mt.Ms0_cell || mt.K1_cell || mt.e_A_cell || mt.Tc_cell || d.T_cell;
}

mmc_status validate(const mmc_chain_desc &d, const mmc_options &o, int idx) {
  const std::string w = "chain " + std::to_string(idx) + ": ";
  const mmc_mesh &m = d.mesh;
  if (m.nx < 1 || m.ny < 1 || m.nz < 1) return fail(MMC_ERR_ARG, w + "mesh extents must be >= 1");
  const long long n = 1LL * m.nx * m.ny * m.nz;
  if (n >= (1LL << 31)) return fail(MMC_ERR_ARG, w + "more than 2^31 cells");
  const int ext[3] = {m.nx, m.ny, m.nz};
  for (int a = 0; a < 3; ++a)
    if (m.periodic[a] && (ext[a] < 2 || ext[a] % 2))
      return fail(MMC_ERR_ARG, w + "a periodic extent must be even and >= 2");
  if (m.demag_images < 0 || m.demag_images > kMaxDemagImages)
    return fail(MMC_ERR_ARG, w + "demag_images must be in [0, " + std::to_string(kMaxDemagImages) + "]");
  for (int a = 0; a < 3; ++a)
    if (!(d.cellsize[a] > 0.0)) return fail(MMC_ERR_ARG, w + "cell size must be > 0");
  const mmc_material &mt = d.material;
  if (!(mt.Ms0 > 0.0) && !mt.Ms0_cell) return fail(MMC_ERR_ARG, w + "Ms0 must be > 0");
  if (!(mt.Tc > 0.0) && !mt.Tc_cell) return fail(MMC_ERR_ARG, w + "Tc must be > 0");
  if (!d.T_cell && !(d.T > 0.0)) return fail(MMC_ERR_ARG, w + "T must be > 0");
  if (d.T_cell)
    for (long long i = 0; i < n; ++i)
      if (!(d.T_cell[i] > 0.0)) return fail(MMC_ERR_ARG, w + "T_cell must be > 0 everywhere");
  if (mt.Ms0_cell)
    for (long long i = 0; i < n; ++i)
      if (!(mt.Ms0_cell[i] > 0.0)) return fail(MMC_ERR_ARG, w + "Ms0_cell must be > 0");
  if (mt.Tc_cell)
    for (long long i = 0; i < n; ++i)
      if (!(mt.Tc_cell[i] > 0.0)) return fail(MMC_ERR_ARG, w + "Tc_cell must be > 0");
  const bool percell = mt.Ms0_cell || mt.K1_cell || mt.e_A_cell || mt.Tc_cell || d.T_cell;
  if (percell && mt.aniso_cubic)
    return fail(MMC_ERR_UNSUPPORTED, w + "cubic anisotropy with per-cell material or temperature");
  if (o.demag) {
    const int P[3] = {pad_len(m.nx, true), pad_len(m.ny, true), pad_len(m.nz, m.nz > 1)};
    for (int a = 0; a < 3; ++a)
      if (P[a] > kMaxFFT) return fail(MMC_ERR_ARG, w + "padded FFT length above 4096");
    if (1LL * P[1] * P[2] > 8192) return fail(MMC_ERR_UNSUPPORTED, w + "padded ny*nz plane above 8192");
  }
  return MMC_OK;
}

// temperature-dependent tables of a chain (Eqs. 7-9, 13 and the m_e scaling
// laws): thermodynamic tables, kT-unit coefficients of ChainDev and, for
// per-cell chains, the per-cell energy table; T_cell (natural order) or the
// scalar T
void apply_temperature(ChainHost &H, ChainDev &D, const mmc_options &o, double Tscalar, const double *T_cell) {
  EnergyCoef &E = H.ecoef;
  const int l1 = H.l1, l2 = H.l2;
  const double *e = H.e;
  H.T = Tscalar;
  if (!H.percell) {
    const double kT = kB * Tscalar;
    H.Tref = Tscalar;
    const Thermo t = thermo(Tscalar, H.Tc, H.mu, H.V, H.Ms0, o.sigma_cap);
    H.me = {t.me}; H.chi = {t.chi}; H.sigma = {t.sigma};
    D.p2 = (float)(t.c2 / kT);
    D.p4 = (float)(t.c4 / kT);
    split_f(t.me2, D.me2h, D.me2l);
    D.sigma = (float)t.sigma;
    D.zee = (float)(H.V * H.Ms0 / kT);
    const double K1T = H.K1 * std::pow(t.me, l1), K2T = H.K2 * std::pow(t.me, l2);
    D.k1 = (float)(H.V * K1T / kT);
    D.k2 = (float)(H.V * K2T / kT);
    for (int a = 0; a < 3; ++a) (&D.wx)[a] = (float)(E.cex[a] / kT);
    D.cdx = (float)(E.cdmi[0] / kT);
    D.cdy = (float)(E.cdmi[1] / kT);
    D.ex = (float)e[0]; D.ey = (float)e[1]; D.ez = (float)e[2];
    E.c2 = t.c2; E.c4 = t.c4; E.me2 = t.me2; E.K1T = K1T; E.K2T = K2T;
    const double len = t.me > 0 ? t.me : rms_len_eq7(Tscalar, H.Tc, H.mu, H.V, H.Ms0);
    H.init_len.assign((size_t)H.ncell, (float)len);
  } else {
    double Tref = 0;
    for (long long i = 0; i < H.ncell; ++i) Tref = std::max(Tref, T_cell ? T_cell[i] : Tscalar);
    H.Tref = Tref;
    const double kTr = kB * Tref;
    for (int a = 0; a < 3; ++a) (&D.wx)[a] = (float)(E.cex[a] / kTr);
    D.cdx = (float)(E.cdmi[0] / kTr);
    D.cdy = (float)(E.cdmi[1] / kTr);
    H.me.assign((size_t)H.ncell, 0); H.chi.assign((size_t)H.ncell, 0); H.sigma.assign((size_t)H.ncell, 0);
    H.etab.assign((size_t)H.ncell * 10, 0.0);
    H.init_len.assign((size_t)H.ncell, 0.f);
    const double cap = o.sigma_cap, mu = H.mu, V = H.V, K2 = H.K2;
    parallel_for(H.ncell, [&](long long i) {
      const double T = T_cell ? T_cell[i] : Tscalar;
      const double Tc = H.Tc_cell.empty() ? H.Tc : H.Tc_cell[(size_t)i];
      const double Ms = H.Ms0_cell.empty() ? H.Ms0 : H.Ms0_cell[(size_t)i];
      const double K1 = H.K1_cell.empty() ? H.K1 : H.K1_cell[(size_t)i];
      const Thermo t = thermo(T, Tc, mu, V, Ms, cap);
      H.me[i] = t.me; H.chi[i] = t.chi; H.sigma[i] = t.sigma;
      double ee[3] = {e[0], e[1], e[2]};
      if (!H.eA_cell.empty()) {
        double n2 = 0;
        for (int a = 0; a < 3; ++a) { ee[a] = H.eA_cell[(size_t)(3 * i + a)]; n2 += ee[a] * ee[a]; }
        n2 = std::sqrt(n2);
        if (!(n2 > 0)) { ee[0] = 0; ee[1] = 0; ee[2] = 1; n2 = 1; }
        for (int a = 0; a < 3; ++a) ee[a] /= n2;
        if (ee[2] < 0) for (int a = 0; a < 3; ++a) ee[a] = -ee[a];
      }
      double *et = &H.etab[10 * i];
      et[0] = t.c2; et[1] = t.c4; et[2] = t.me2; et[3] = Ms;
      et[4] = K1 * std::pow(t.me, l1); et[5] = K2 * std::pow(t.me, l2);
      et[6] = ee[0]; et[7] = ee[1]; et[8] = ee[2]; et[9] = kB * T;
      H.init_len[i] = (float)(t.me > 0 ? t.me : 0.3);
    });
  }
}

// tables of one chain (host); a batch in which any chain has per-cell inputs
// gives every chain per-cell tables (force_percell), since one sweep launch
// reads all chains of the batch the same way
void build_chain(ChainHost &H, ChainDev &D, const mmc_chain_desc &d, const mmc_options &o, int idx,
                 bool force_percell) {
  const mmc_material &mt = d.material;
  H.mesh = d.mesh;
  for (int a = 0; a < 3; ++a) H.h[a] = d.cellsize[a];
  H.V = H.h[0] * H.h[1] * H.h[2];
  H.T = d.T; H.Tc = mt.Tc; H.Ms0 = mt.Ms0; H.K1 = mt.K1; H.K2 = mt.K2;
  H.mu = mt.mu_atom > 0 ? mt.mu_atom : muB;
  H.cubic = mt.aniso_cubic;
  H.percell = has_percell(d) || force_percell;
  const int nx = d.mesh.nx, ny = d.mesh.ny, nz = d.mesh.nz;
  H.ncell = 1LL * nx * ny * nz;
  const int hx = (nx + 1) / 2;
  H.slots = 1LL * hx * ny * nz;

  std::memset(&D, 0, sizeof(D));
  D.nx = nx; D.ny = ny; D.nz = nz; D.hx = hx; D.nrows = ny * nz;
  D.pbc = (d.mesh.periodic[0] ? 1 : 0) | (d.mesh.periodic[1] ? 2 : 0) | (d.mesh.periodic[2] ? 4 : 0);
  D.chain = o.chain_base + idx;
  D.ncell = H.ncell;
  divmagic((unsigned)hx, D.hx_m, D.hx_l);
  divmagic((unsigned)ny, D.ny_m, D.ny_l);
  divmagic((unsigned)nx, D.nx_m, D.nx_l);
  D.h_off = -1; D.t_off = -1; D.ms_off = -1;
  D.Bx = (float)d.B[0]; D.By = (float)d.B[1]; D.Bz = (float)d.B[2];
  D.gscale = (float)(mt.grain ? mt.grain_exch_scale : 1.0);
  D.Ms0 = (float)mt.Ms0;
  D.Ms0d = mt.Ms0;
  double e[3] = {mt.e_A[0], mt.e_A[1], mt.e_A[2]};
  double en = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  if (!(en > 0)) { e[0] = 0; e[1] = 0; e[2] = 1; en = 1; }
  for (int a = 0; a < 3; ++a) e[a] /= en;
  if (e[2] < 0) for (int a = 0; a < 3; ++a) e[a] = -e[a];   // uniaxial: e and -e are the same axis
  int flags = 0;
  if (mt.grain) flags |= F_GRAIN;
  if (mt.D0 != 0.0) flags |= F_DMI;
  if (mt.aniso_cubic) flags |= F_CUBIC;
  else if (mt.K1 != 0.0 || mt.K2 != 0.0 || mt.K1_cell) flags |= F_ANIS;
  if (o.demag) flags |= F_DEMAG;
  D.flags = flags;
  const int l1 = mt.aniso_cubic ? 10 : 3, l2 = mt.aniso_cubic ? 21 : 10;

  // energy coefficients (J)
  EnergyCoef &E = H.ecoef;
  std::memset(&E, 0, sizeof(E));
  for (int a = 0; a < 3; ++a) E.cex[a] = H.V * mt.A0 / (H.h[a] * H.h[a]);
  for (int a = 0; a < 2; ++a) E.cdmi[a] = H.V * mt.D0 / H.h[a];
  E.V = H.V;
  E.cubic = mt.aniso_cubic;
  for (int a = 0; a < 3; ++a) { E.B[a] = d.B[a]; E.e[a] = e[a]; }
  E.Ms0 = mt.Ms0;

  for (int a = 0; a < 3; ++a) H.e[a] = e[a];
  H.l1 = l1;
  H.l2 = l2;
  if (mt.Ms0_cell) H.Ms0_cell.assign(mt.Ms0_cell, mt.Ms0_cell + H.ncell);
  if (mt.K1_cell) H.K1_cell.assign(mt.K1_cell, mt.K1_cell + H.ncell);
  if (mt.Tc_cell) H.Tc_cell.assign(mt.Tc_cell, mt.Tc_cell + H.ncell);
  if (mt.e_A_cell) H.eA_cell.assign(mt.e_A_cell, mt.e_A_cell + 3 * H.ncell);
  apply_temperature(H, D, o, d.T, d.T_cell);
  if (mt.grain) {
    H.grain.resize((size_t)H.ncell);
    for (long long i = 0; i < H.ncell; ++i) H.grain[i] = (float)mt.grain[i];
  }
}

// split-layout index of natural cell (i, row)
inline long long split_index(const ChainDev &D, int i, int row) {
  const int j = row % D.ny, k = row / D.ny;
  const int col = (i + j + k) & 1;
  return (long long)col * D.nrows * D.hx + (long long)row * D.hx + (i >> 1);
}

// per-cell tables of a chain in the split layout: 3 float4 arrays of 2 S entries
// ({p2, p4, m_e^2, sigma}, {zee, k1, k2, T_ref / T}, {e_A}) and Ms0 per cell
void fill_percell_tables(const ChainHost &H, const ChainDev &D, float4 *tab, float *ms, float *ms_lo) {
  const long long S = H.slots;
  for (int row = 0; row < D.nrows; ++row)
    for (int i = 0; i < D.nx; ++i) {
      const long long nat = i + (long long)D.nx * row;
      const long long si = split_index(D, i, row);
      const double *et = &H.etab[10 * nat];
      const double kT = et[9];
      const float bs = (float)(kB * H.Tref / kT);
      tab[si] = make_float4((float)(et[0] / kT), (float)(et[1] / kT), (float)et[2], (float)H.sigma[(size_t)nat]);
      tab[2 * S + si] =
          make_float4((float)(H.V * et[3] / kT), (float)(H.V * et[4] / kT), (float)(H.V * et[5] / kT), bs);
      // m_e^2 as a float-float pair (high part in the first table, low part here)
      tab[4 * S + si] = make_float4((float)et[6], (float)et[7], (float)et[8], (float)(et[2] - (double)(float)et[2]));
      ms[si] = (float)et[3];
      ms_lo[si] = (float)(et[3] - (double)ms[si]);
    }
}

// block tables of the 2D kernels: block -> chain id (ids[t] for the t-th chain of
// `table`) and, per chain id, its first block
mmc_status build_il_tables(mmc_ctx *c, IlTables &T, const std::vector<ChainDev> &table, const std::vector<int> &ids,
                           int nid, int E, bool fp64) {
  const size_t csz = fp64 ? 16 : 8;
  int maxPx = 1, maxPy = 1;
  for (const ChainDev &D : table) {
    if (D.Pz != 1 || 3 * D.Px > E || 3 * D.Py > E) return MMC_OK;   // T.ok stays false
    maxPx = std::max(maxPx, D.Px);
    maxPy = std::max(maxPy, D.Py);
  }
  std::vector<int> rc, colc;
  std::vector<long long> rf((size_t)nid + 1, 0), colf((size_t)nid + 1, 0);
  for (size_t t = 0; t < table.size(); ++t) {
    const ChainDev &D = table[t];
    const int np = E / (3 * D.Px);
    const int nb = ((D.nrows + 1) / 2 + np - 1) / np;
    rf[(size_t)ids[t]] = (long long)rc.size();
    for (int b = 0; b < nb; ++b) rc.push_back(ids[t]);
    const int CC = E / (3 * D.Py);
    const int nc = D.Sx / CC;
    colf[(size_t)ids[t]] = (long long)colc.size();
    for (int b = 0; b < nc; ++b) colc.push_back(ids[t]);
  }
  MMC_TRY(upload(c, &T.rows_chain, rc));
  MMC_TRY(upload(c, &T.rows_first, rf));
  MMC_TRY(upload(c, &T.cols_chain, colc));
  MMC_TRY(upload(c, &T.cols_first, colf));
  T.rows_blocks = (int)rc.size();
  T.cols_blocks = (int)colc.size();
  const int Ep = il_padded_of(E);
  T.rows_smem = (size_t)(Ep + maxPx) * csz;
  T.cols_smem = (size_t)(Ep + maxPy) * csz;
  T.inv_smem = (size_t)(Ep + maxPx) * csz;
  T.ok = true;
  return MMC_OK;
}

// The spectrum buffer of the warp-transform path as a 2D FP32 tensor: one row per
// tile of four rows (kW32Tile complex values, 4160 floats, 16,640 bytes), `tiles`
// rows; boxes of 8 floats (one kx of a tile) x 128 tiles (a 512-row column).
// The encoder is the driver's, looked up through the runtime (no link to the
// driver library).
static bool encode_spec_map(CUtensorMap *map, void *spec, long long tiles) {
  using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  // looked up once (thread-safe initialization of a function-local static)
  static const Encode enc = []() -> Encode {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<Encode>(fn);
  }();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * kW32Tile), (cuuint64_t)tiles};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * kW32Tile) * sizeof(float)};
  const cuuint32_t box[2] = {8, 128};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Plan of the demag kernels over `chains`.  single: the plan carries its own
// chain table and spectrum buffer (chain ids are positions in `chains`);
// otherwise it indexes the context's chain table by global chain id and uses the
// spectrum buffer shared_spec when given (chain offsets are the batch's).
mmc_status build_demag_plan(mmc_ctx *c, DemagPlan &P, const std::vector<int> &chains, bool fp64,
                            bool single, void *shared_spec = nullptr) {
  const size_t csz = fp64 ? 16 : 8;
  std::vector<int> ids(chains.size());
  for (size_t t = 0; t < chains.size(); ++t) ids[t] = single ? (int)t : chains[t];
  const int nid = single ? (int)chains.size() : c->nchains;
  std::vector<ChainDev> table;
  long long spec_elems = 0;
  int maxPx = 1, maxPyPz = 1;
  for (int ci : chains) {
    ChainDev D = c->ch[ci];
    if (single) {
      D.s_off = spec_elems;
    }
    spec_elems += 3LL * spectrum_rows(D) * D.Sx;
    table.push_back(D);
    maxPx = std::max(maxPx, D.Px);
    maxPyPz = std::max(maxPyPz, D.Py * D.Pz);
  }
  if (single) {
    MMC_TRY(upload(c, &P.d_ch, table));
  } else {
    P.d_ch = c->d_ch;
  }
  // 2D chains use the interleaved radix-16 kernels: E elements per block,
  // 3 sequences per row pair (np = E / (3 Px)) or 3 components per column
  // (CC = E / (3 Py))
  const int E = il_elements(fp64);
  // float-float convolution of the sweep's field (energies keep FP64 single-chain
  // plans): always the generic kernels
  const bool ffp = fp64 && !single && c->opt.demag_fp64 == 2 && c->d_nhatff != nullptr;
  bool il = !ffp;
  for (const ChainDev &D : table)
    if (D.Pz != 1 || 3 * D.Px > E || 3 * D.Py > E) il = false;
  std::vector<int> rc, colc;
  std::vector<long long> rf((size_t)nid + 1, 0), colf((size_t)nid + 1, 0);
  size_t rsmem = 0, csmem = 0;
  int T = 384, Tc = 384, cc = 1;
  if (il) {
    for (size_t t = 0; t < table.size(); ++t) {
      const ChainDev &D = table[t];
      const int np = E / (3 * D.Px);
      const int nb = ((D.nrows + 1) / 2 + np - 1) / np;
      rf[(size_t)ids[t]] = (long long)rc.size();
      for (int b = 0; b < nb; ++b) rc.push_back(ids[t]);
      const int CC = E / (3 * D.Py);
      const int nc = D.Sx / CC;
      colf[(size_t)ids[t]] = (long long)colc.size();
      for (int b = 0; b < nc; ++b) colc.push_back(ids[t]);
    }
    // data block (padded capacity), then the block's twiddle table (Px entries for
    // the row kernels, Py for the column kernel)
    const int Ep = il_padded_elements(fp64);
    rsmem = (size_t)(Ep + maxPx) * csz;
    csmem = (size_t)(Ep + maxPyPz) * csz;
    P.inv_smem = (size_t)(Ep + maxPx) * csz;
  } else {
    const int Gmax = std::max(maxPx / 8, 1);
    T = std::min(512, std::max(64, 3 * Gmax));
    T = (T + 31) / 32 * 32;
    if (T < Gmax) T = Gmax;
    for (size_t t = 0; t < table.size(); ++t) {
      const ChainDev &D = table[t];
      const int G = std::max(D.Px / 8, 1);
      const int np = std::max(1, std::min(8, T / (3 * G)));
      const int pairs = (D.nrows + 1) / 2;
      const int nb = (pairs + np - 1) / np;
      rf[(size_t)ids[t]] = (long long)rc.size();
      for (int b = 0; b < nb; ++b) rc.push_back(ids[t]);
      rsmem = std::max(rsmem, (size_t)3 * np * D.Px * csz);
    }
    cc = 8;
    while (cc > 1 && (size_t)3 * cc * maxPyPz * csz > 100 * 1024) cc >>= 1;
    csmem = (size_t)3 * cc * maxPyPz * csz;
    if (csmem > 200 * 1024) return fail(MMC_ERR_UNSUPPORTED, "column FFT plane too large for shared memory");
    int Gy = 1;
    for (size_t t = 0; t < table.size(); ++t) {
      const ChainDev &D = table[t];
      Gy = std::max(Gy, std::max(D.Py / 8, std::max(D.Pz / 8, 1)));
      const int nb = (D.Px / 2 + 1 + cc - 1) / cc;
      colf[(size_t)ids[t]] = (long long)colc.size();
      for (int b = 0; b < nb; ++b) colc.push_back(ids[t]);
    }
    Tc = std::min(512, std::max(128, 3 * cc * Gy));
    Tc = (Tc + 31) / 32 * 32;
    if (Tc < Gy) Tc = Gy;
  }
  P.il2d = il;
  MMC_TRY(upload(c, &P.rows_chain, rc));
  MMC_TRY(upload(c, &P.rows_first, rf));
  MMC_TRY(upload(c, &P.cols_chain, colc));
  MMC_TRY(upload(c, &P.cols_first, colf));
  P.rows_blocks = (int)rc.size();
  P.rows_threads = T;
  P.rows_smem = rsmem;
  P.cols_blocks = (int)colc.size();
  P.cols_threads = Tc;
  P.cols_cc = cc;
  P.cols_smem = csmem;
  P.fp64 = fp64;
  P.ff = ffp;
  P.nchain_table = nid;
  if (il && !fp64) MMC_TRY(build_il_tables(c, P.small, table, ids, nid, il_elements_small(), false));
  if (il && !fp64 && !single) {
    // warp-transform path: every chain on a 1024 x 1024 padded grid; one row block
    // per tile of four rows, one column block per kx = 0..512
    bool ok = !table.empty();
    for (const ChainDev &D : table) ok = ok && w32_chain(D) && c->specs[(size_t)D.spec].d32t != nullptr;
    if (ok) {
      std::vector<int> rc2, cc2;
      std::vector<long long> rf2((size_t)nid + 1, 0), cf2((size_t)nid + 1, 0);
      for (size_t t = 0; t < table.size(); ++t) {
        const ChainDev &D = table[t];
        rf2[(size_t)ids[t]] = (long long)rc2.size();
        for (long long b = 0; b < spectrum_rows(D) / 4; ++b) rc2.push_back(ids[t]);
        cf2[(size_t)ids[t]] = (long long)cc2.size();
        for (int b = 0; b < D.Px / 2 + 1; ++b) cc2.push_back(ids[t]);
      }
      MMC_TRY(upload(c, &P.w32.rows_chain, rc2));
      MMC_TRY(upload(c, &P.w32.rows_first, rf2));
      MMC_TRY(upload(c, &P.w32.cols_chain, cc2));
      MMC_TRY(upload(c, &P.w32.cols_first, cf2));
      P.w32.rows_blocks = (int)rc2.size();
      P.w32.cols_blocks = (int)cc2.size();
      P.w32.ok = true;
    }
  }
  {
    int v = c->opt.fft_variant >= 1 && c->opt.fft_variant <= 4 ? c->opt.fft_variant
            : (c->tuned_variant ? c->tuned_variant : 1);
    if (v == 3 && !P.small.ok) v = 1;
    if (v == 4 && !P.w32.ok) v = 1;
    P.fft_variant = v;
  }
  if (shared_spec) {
    P.spec = shared_spec;
  } else {
    MMC_TRY(dalloc(c, &P.spec, (size_t)spec_elems * csz));
    CUDA_TRY(cudaMemset(P.spec, 0, (size_t)spec_elems * csz));   // padding columns stay defined
  }
  if (P.w32.ok) {
    // the tensor spans the whole buffer (a shared one holds every chain of the batch)
    long long tot = spec_elems;
    if (shared_spec) {
      tot = 0;
      for (const ChainDev &D : c->ch) tot += 3LL * spectrum_rows(D) * D.Sx;
    }
    if (tot % kW32Tile != 0 || !encode_spec_map(&P.tmap_spec, P.spec, tot / kW32Tile)) {
      P.w32.ok = false;
      if (P.fft_variant == 4) P.fft_variant = 1;
    }
  }
  P.ready = true;
  return MMC_OK;
}

DemagLaunch make_demag_launch(mmc_ctx *c, const DemagPlan &P, float4 *heff, double *Hd, int Hd_chain) {
  DemagLaunch D;
  D.chains = P.d_ch;
  D.m = c->d_m;
  D.tab = c->d_tab;
  D.ms = c->d_ms;
  D.ms_lo = c->d_ms_lo;
  D.spec = P.spec;
  D.nhat = P.ff ? (const void *const *)c->d_nhatff
           : P.fp64 ? (const void *const *)c->d_nhat64 : (const void *const *)c->d_nhat32;
  D.twiddle = P.ff ? c->d_twff : P.fp64 ? c->d_tw64 : c->d_tw32;
  D.ff = P.ff;
  D.heff = heff;
  D.Hd = Hd;
  D.Hd_chain = Hd_chain;
  D.rows_chain = P.rows_chain;
  D.rows_first = P.rows_first;
  D.rows_blocks = P.rows_blocks;
  D.rows_threads = P.rows_threads;
  D.rows_smem = P.rows_smem;
  D.cols_chain = P.cols_chain;
  D.cols_first = P.cols_first;
  D.cols_blocks = P.cols_blocks;
  D.cols_threads = P.cols_threads;
  D.cols_per_block = P.cols_cc;
  D.cols_smem = P.cols_smem;
  D.ev = nullptr;
  D.m_nat = nullptr;
  D.Ms_override = 0.0;
  D.il2d = P.il2d;
  D.fft_variant = P.fft_variant;
  D.inv_smem = P.inv_smem;
  D.w32 = false;
  D.err = c->d_err;
  D.ck = c->d_check;
  D.nchains = P.nchain_table;
  D.nhatT = (const void *const *)c->d_nhat32t;
  D.tw1024 = c->d_tw1024;
  D.tmap_spec = &P.tmap_spec;
  if (P.il2d && P.fft_variant == 4 && P.w32.ok && !P.fp64) {
    D.w32 = true;
    D.rows_chain = P.w32.rows_chain; D.rows_first = P.w32.rows_first; D.rows_blocks = P.w32.rows_blocks;
    D.cols_chain = P.w32.cols_chain; D.cols_first = P.w32.cols_first; D.cols_blocks = P.w32.cols_blocks;
  }
  if (P.il2d && P.fft_variant == 3 && P.small.ok) {
    D.rows_chain = P.small.rows_chain; D.rows_first = P.small.rows_first; D.rows_blocks = P.small.rows_blocks;
    D.cols_chain = P.small.cols_chain; D.cols_first = P.small.cols_first; D.cols_blocks = P.small.cols_blocks;
    D.rows_smem = P.small.rows_smem; D.cols_smem = P.small.cols_smem; D.inv_smem = P.small.inv_smem;
  }
  return D;
}

mmc_status single_plan(mmc_ctx *c, int chain, bool fp64, DemagPlan **out) {
  std::vector<DemagPlan> &v = c->single[fp64 ? 1 : 0];
  if ((int)v.size() < c->nchains) v.resize(c->nchains);
  DemagPlan &P = v[chain];
  if (!P.ready) MMC_TRY(build_demag_plan(c, P, std::vector<int>{chain}, fp64, true));
  *out = &P;
  return MMC_OK;
}

SweepLaunch sweep_launch(mmc_ctx *c, int color, unsigned off, unsigned key0, unsigned key1) {
  SweepLaunch P;
  P.chains = c->d_ch;
  P.st = c->d_st;
  P.blk_desc = c->d_sw_desc;
  P.blk_base = 0;
  P.nblocks = c->sw_blocks;
  P.m = c->d_m;
  P.heff = c->d_heff;
  P.tab = c->d_tab;
  P.sweep_base = c->d_sweep_base;
  P.sweep_off = off;
  P.key0 = key0;
  P.key1 = key1;
  P.color = color;
  P.percell = c->any_percell;
  P.omc_override = -1.f;
  P.dec_dbg = nullptr;
  P.acc_dbg = nullptr;
  P.nstripes = 1;
  P.stripe = 0;
  P.flat = c->all_flat;
  P.band = c->band;
  P.items = c->d_items;
  P.i0 = 0;
  P.i1 = c->band ? c->item_first.back() : 0;
  P.band_grid = c->band_grid;
  P.stage_own = c->stage_own;
  P.stage_other = c->stage_other;
  P.max_polls = c->opt.wait_polls > 0 ? (unsigned)c->opt.wait_polls : (1u << 22);
  P.err = c->d_err;
  P.wait_test = c->opt.wait_test;
  P.ck = c->d_check;
  P.blk_total = c->sw_blocks;
  P.nchains = c->nchains;
  P.nitems = c->band ? c->item_first.back() : 0;
  return P;
}

// bands of rows per sublattice pass (the demag field recomputed before each)
int pass_bands(const mmc_ctx *c) { return c->any_demag && c->opt.demag_stripes > 1 ? c->opt.demag_stripes : 1; }

ObsLaunch obs_launch(mmc_ctx *c, int accumulate) {
  ObsLaunch P;
  P.chains = c->d_ch;
  P.st = c->d_st;
  P.blk_chain = c->d_obs_chain;
  P.blk_first = c->d_obs_first;
  P.nblocks = c->obs_blocks;
  P.nchains = c->nchains;
  P.m = c->d_m;
  P.part = c->d_part;
  P.hist = accumulate ? c->d_hist_acc : c->d_hist_cur;
  P.bins = c->opt.hist_bins;
  P.scale = (float)c->opt.hist_bins / (float)c->opt.hist_max;
  P.out = c->d_obs_out;
  P.accumulate = accumulate;
  return P;
}

// optional per-kernel event timing (mmc_phase_times)
struct PhaseTimer {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<int, int>>> marks;   // (kind, (ev0, ev1))
  size_t used = 0;
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
};

void issue_demag(mmc_ctx *c, PhaseTimer *pt = nullptr) {
  Launch L = c->L();
  if (!c->cf.empty()) {
    const void *const *nh = c->opt.demag_fp64 ? (const void *const *)c->d_nhat64 : (const void *const *)c->d_nhat32;
    for (auto &G : c->cf) {
      cudaEvent_t ev[4];
      cudaEvent_t *evp = nullptr;
      if (pt) {
        int idx[4];
        for (int k = 0; k < 4; ++k) { idx[k] = (int)pt->used; ev[k] = pt->next(); }
        for (int k = 0; k < 3; ++k) pt->marks.push_back({k, {idx[k], idx[k + 1]}});
        evp = ev;
      }
      launch_cufft_group(L, G, c->d_ch, c->d_m, c->d_ms, c->d_tab, c->d_heff, nullptr, -1, nh, evp);
    }
    return;
  }
  DemagLaunch D = make_demag_launch(c, c->batch_plan, c->d_heff, nullptr, -1);
  cudaEvent_t ev[4];
  if (pt) {
    int idx[4];
    for (int k = 0; k < 4; ++k) { idx[k] = (int)pt->used; ev[k] = pt->next(); }
    for (int k = 0; k < 3; ++k) pt->marks.push_back({k, {idx[k], idx[k + 1]}});
    D.ev = ev;
  }
  launch_demag(L, D, c->batch_plan.fp64);
}

template <typename F>
void timed(mmc_ctx *c, PhaseTimer *pt, int kind, F fn) {
  if (!pt) { fn(); return; }
  const int i0 = (int)pt->used;
  cudaEventRecord(pt->next(), c->stream);
  fn();
  const int i1 = (int)pt->used;
  cudaEventRecord(pt->next(), c->stream);
  pt->marks.push_back({kind, {i0, i1}});
}

// the iteration of batches on the warp-transform demag path with uniform
// one-cell-thick chains fuses the red pass with the inverse row transforms
// (k_w32_rows_inv_red) and the black pass with the next iteration's forward row
// transforms (k_w32_black_rows_fwd): a block of k iterations is the forward rows
// of the current state, then k times {columns, inverse rows + red pass, black
// pass + forward rows}
bool fused_path(const mmc_ctx *c) {
  return c->opt.fuse_passes && c->any_demag && c->cf.empty() && !c->batch_plan.fp64 &&
         c->batch_plan.fft_variant == 4 && c->batch_plan.w32.ok && c->all_flat && !c->any_percell && !c->band &&
         !c->opt.demag_per_pass && pass_bands(c) == 1;
}

// k fused iterations of the chains of plan / blocks [b0, b0 + nb) on L
void issue_fused(mmc_ctx *c, const Launch &L, const DemagPlan &plan, int k, unsigned key0, unsigned key1,
                 int sample_every, uint64_t start, PhaseTimer *pt) {
  const DemagLaunch D = make_demag_launch(c, plan, c->d_heff, nullptr, -1);
  const auto tm = [&](int kind, const std::function<void()> &fn) {
    if (!pt) { fn(); return; }
    const int i0 = (int)pt->used;
    cudaEventRecord(pt->next(), L.stream);
    fn();
    const int i1 = (int)pt->used;
    cudaEventRecord(pt->next(), L.stream);
    pt->marks.push_back({kind, {i0, i1}});
  };
  tm(0, [&] { launch_w32_stage(L, D, 0); });
  for (int off = 0; off < k; ++off) {
    tm(1, [&] { launch_w32_stage(L, D, 1); });
    const SweepLaunch red = sweep_launch(c, 0, (unsigned)off, key0, key1);
    tm(7, [&] { launch_w32_rows_inv_red(L, D, red); });
    const SweepLaunch blk = sweep_launch(c, 1, (unsigned)off, key0, key1);
    tm(6, [&] { launch_w32_black_rows_fwd(L, D, blk); });
    if (sample_every > 0 && (start + off + 1) % (uint64_t)sample_every == 0) {
      Trace t("observables");
      tm(4, [&] { launch_obs(L, obs_launch(c, 1)); });
    }
  }
}

// k sweeps starting at global sweep index `start` (device base == start)
void issue_block(mmc_ctx *c, int k, unsigned key0, unsigned key1, int sample_every, uint64_t start,
                 PhaseTimer *pt = nullptr) {
  Launch L = c->L();
  if (fused_path(c)) {
    if (!c->groups.empty() && !pt && sample_every == 0) {
      cudaEventRecord(c->ev_fork, c->stream);
      for (auto &g : c->groups) {
        cudaStreamWaitEvent(g.stream, c->ev_fork, 0);
        Launch Lg{g.stream, &c->launches};
        issue_fused(c, Lg, g.plan, k, key0, key1, 0, start, nullptr);
        cudaEventRecord(g.done, g.stream);
        cudaStreamWaitEvent(c->stream, g.done, 0);
      }
    } else {
      issue_fused(c, L, c->batch_plan, k, key0, key1, sample_every, start, pt);
    }
    const int adapt_now = ((start + k) % 100 == 0) ? 1 : 0;
    Trace t("advance");
    timed(c, pt, 5, [&] {
      launch_advance(L, c->d_st, c->nchains, (unsigned)k, c->d_sweep_base, adapt_now, c->opt.adapt, 1.f, 180.f);
    });
    return;
  }
  if (!c->groups.empty() && !pt && sample_every == 0) {
    // fork: every group runs its k iterations on its own stream (the chains of
    // different groups never interact), join before the window step
    cudaEventRecord(c->ev_fork, c->stream);
    for (auto &g : c->groups) {
      cudaStreamWaitEvent(g.stream, c->ev_fork, 0);
      Launch Lg{g.stream, &c->launches};
      const int b0 = (int)c->sw_first[(size_t)g.c0], nb = (int)(c->sw_first[(size_t)g.c1] - b0);
      const int nbands = pass_bands(c);
      for (int off = 0; off < k; ++off) {
        for (int color = 0; color < 2; ++color) {
          for (int band = 0; band < nbands; ++band) {
            if (c->any_demag && ((color == 0 && band == 0) || c->opt.demag_per_pass || nbands > 1))
              launch_demag(Lg, make_demag_launch(c, g.plan, c->d_heff, nullptr, -1), g.plan.fp64);
            SweepLaunch P = sweep_launch(c, color, (unsigned)off, key0, key1);
            P.blk_base = b0;
            P.nblocks = nb;
            if (c->band) {
              P.i0 = c->item_first[(size_t)g.c0];
              P.i1 = c->item_first[(size_t)g.c1];
            }
            P.nstripes = nbands;
            P.stripe = band;
            launch_sweep_pass(Lg, P);
          }
        }
      }
      cudaEventRecord(g.done, g.stream);
      cudaStreamWaitEvent(c->stream, g.done, 0);
    }
    const int adapt_now = ((start + k) % 100 == 0) ? 1 : 0;
    launch_advance(L, c->d_st, c->nchains, (unsigned)k, c->d_sweep_base, adapt_now, c->opt.adapt, 1.f, 180.f);
    return;
  }
  const int nbands = pass_bands(c);
  for (int off = 0; off < k; ++off) {
    for (int color = 0; color < 2; ++color) {
      for (int band = 0; band < nbands; ++band) {
        if (c->any_demag && ((color == 0 && band == 0) || c->opt.demag_per_pass || nbands > 1)) {
          Trace t("demag");
          issue_demag(c, pt);
        }
        Trace t(color == 0 ? "pass red" : "pass black");
        SweepLaunch P = sweep_launch(c, color, (unsigned)off, key0, key1);
        P.nstripes = nbands;
        P.stripe = band;
        timed(c, pt, 3, [&] { launch_sweep_pass(L, P); });
      }
    }
    if (sample_every > 0 && (start + off + 1) % (uint64_t)sample_every == 0) {
      Trace t("observables");
      timed(c, pt, 4, [&] { launch_obs(L, obs_launch(c, 1)); });
    }
  }
  const int adapt_now = ((start + k) % 100 == 0) ? 1 : 0;
  Trace t("advance");
  timed(c, pt, 5, [&] {
    launch_advance(L, c->d_st, c->nchains, (unsigned)k, c->d_sweep_base, adapt_now, c->opt.adapt, 1.f, 180.f);
  });
}

mmc_status check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MMC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return MMC_OK;
}

mmc_status sweep_impl(mmc_ctx *c, int64_t n, uint64_t seed, int sample_every) {
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (n < 0) return fail(MMC_ERR_ARG, "negative sweep count");
  if (sample_every < 0) return fail(MMC_ERR_ARG, "negative sample interval");
  const unsigned key0 = (unsigned)(seed & 0xffffffffu), key1 = (unsigned)(seed >> 32);
  const bool graph_ok = c->opt.use_graphs && (sample_every == 0 || 100 % sample_every == 0);
  while (n > 0) {
    const int k = (int)std::min<int64_t>(n, 100 - (int64_t)(c->host_sweep % 100));
    if (k == 100 && graph_ok) {
      GraphEntry *g = nullptr;
      for (auto &e : c->graphs)
        if (e.key0 == key0 && e.key1 == key1 && e.sample_every == sample_every) g = &e;
      if (!g) {
        GraphEntry e;
        e.key0 = key0; e.key1 = key1; e.sample_every = sample_every;
        const long long before = c->launches;
        CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        issue_block(c, 100, key0, key1, sample_every, c->host_sweep);
        cudaGraph_t graph;
        cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
        if (ce != cudaSuccess) return fail(MMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        e.launches = c->launches - before;
        c->launches = before;
        ce = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(MMC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        c->graphs.push_back(e);
        g = &c->graphs.back();
      }
      {
        Trace t("graph: 100 iterations");
        CUDA_TRY(cudaGraphLaunch(g->exec, c->stream));
      }
      c->launches += g->launches;
    } else {
      issue_block(c, k, key0, key1, sample_every, c->host_sweep);
      MMC_TRY(check_launch());
    }
    c->host_sweep += (uint64_t)k;
    n -= k;
  }
  c->heff_stale = true;
  c->obs_fresh = false;
  return MMC_OK;
}

// ---------------------------------------------------------------------------
// Autotuning record cache: one line per tuned problem, "key fft_variant groups",
// in the file named by MMC_TUNE_CACHE (an empty value or "off" disables it), by
// default $XDG_CACHE_HOME/mmc_gb300/tune.txt or ~/.cache/mmc_gb300/tune.txt.
// The key is the GPU name and a 64-bit FNV-1a hash of everything the picks
// depend on: the chains' extents, periodicity, demag images and per-cell flag,
// and the options that select kernels.  A later line wins.
std::string tune_cache_path() {
  const char *e = std::getenv("MMC_TUNE_CACHE");
  if (e) {
    const std::string v(e);
    return (v.empty() || v == "off") ? std::string() : v;
  }
  const char *x = std::getenv("XDG_CACHE_HOME");
  const char *h = std::getenv("HOME");
  if (x && *x) return std::string(x) + "/mmc_gb300/tune.txt";
  if (h && *h) return std::string(h) + "/.cache/mmc_gb300/tune.txt";
  return std::string();
}

std::string tune_key(const mmc_ctx *c) {
  std::ostringstream d;
  d << "v1|n" << c->nchains << "|fp64 " << c->opt.demag_fp64 << "|cufft " << c->opt.demag_cufft << "|demag "
    << c->opt.demag << "|pp " << c->opt.demag_per_pass << "|st " << c->opt.demag_stripes << "|tiles "
    << c->opt.sweep_tiles << "|fuse " << c->opt.fuse_passes;
  for (int i = 0; i < c->nchains; ++i) {
    const mmc_mesh &m = c->hc[i].mesh;
    d << "|" << m.nx << "x" << m.ny << "x" << m.nz << "p" << m.periodic[0] << m.periodic[1] << m.periodic[2] << "i"
      << m.demag_images << "c" << (c->hc[i].percell ? 1 : 0);
  }
  const std::string str = d.str();
  unsigned long long hsh = 1469598103934665603ULL;
  for (unsigned char ch : str) {
    hsh ^= ch;
    hsh *= 1099511628211ULL;
  }
  int dev = 0;
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char &ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  char buf[32];
  std::snprintf(buf, sizeof(buf), "%016llx", hsh);
  return name + ":" + buf;
}

bool tune_cache_read(const std::string &path, const std::string &key, int &fft, int &groups) {
  std::ifstream f(path);
  if (!f) return false;
  bool found = false;
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream in(line);
    std::string k;
    int a = 0, b = 0;
    if ((in >> k >> a >> b) && k == key) {
      fft = a;
      groups = b;
      found = true;
    }
  }
  return found;
}

void tune_cache_write(const std::string &path, const std::string &key, int fft, int groups) {
  std::error_code ec;
  const std::filesystem::path p(path);
  if (p.has_parent_path()) std::filesystem::create_directories(p.parent_path(), ec);
  std::ofstream f(path, std::ios::app);
  if (f) f << key << " " << fft << " " << groups << "\n";
}

void free_groups(mmc_ctx *c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto &g : c->groups) {
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  c->groups.clear();
}

// G groups of contiguous chains with about equal cell counts, each with its own
// stream and demag plan (over the batch's spectrum buffer); G <= 1: no groups
mmc_status make_groups(mmc_ctx *c, int G) {
  free_groups(c);
  const int nchains = c->nchains;
  G = std::min(G, nchains);
  if (G <= 1) return MMC_OK;
  long long total = 0;
  for (int i = 0; i < nchains; ++i) total += c->hc[i].ncell;
  int start = 0;
  long long done = 0;
  for (int gi = 0; gi < G; ++gi) {
    int end = start + 1;
    const long long target = total * (gi + 1) / G;
    long long acc = done + c->hc[start].ncell;
    while (end < nchains - (G - 1 - gi) && acc + c->hc[end].ncell / 2 <= target) acc += c->hc[end++].ncell;
    if (gi == G - 1) { end = nchains; acc = total; }
    mmc_ctx::ChainGroup g;
    g.c0 = start;
    g.c1 = end;
    c->groups.push_back(g);
    start = end;
    done = acc;
  }
  if (!c->ev_fork) CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  for (auto &g : c->groups) {
    CUDA_TRY(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
    if (c->opt.demag) {
      std::vector<int> ids;
      for (int i = g.c0; i < g.c1; ++i) ids.push_back(i);
      MMC_TRY(build_demag_plan(c, g.plan, ids, c->opt.demag_fp64 != 0, false, c->batch_plan.spec));
    }
  }
  return MMC_OK;
}

mmc_status serial_prepare(mmc_ctx *c) {
  if (c->serial_ready) return MMC_OK;
  if (c->any_demag) {
    std::vector<float *> ptrs;
    std::vector<int4> dims;
    for (auto &ss : c->specs) {
      // offsets up to n - 1 per axis: P / 2 >= n on padded axes, P = n on circular ones
      const int ox = ss.pd.circ[0] ? ss.Px : std::max(ss.Px / 2, 1);
      const int oy = ss.pd.circ[1] ? ss.Py : std::max(ss.Py / 2, 1);
      const int oz = ss.pd.circ[2] ? ss.Pz : std::max(ss.Pz / 2, 1);
      std::vector<double> oct;
      demag_octant(ss.h, ox, oy, oz, oct, ss.pd);
      const size_t n = (size_t)ox * oy * oz;
      std::vector<float> soa(6 * n);
      for (size_t q = 0; q < n; ++q)
        for (int k = 0; k < 6; ++k) soa[k * n + q] = (float)oct[6 * q + k];
      float *d = nullptr;
      MMC_TRY(upload(c, &d, soa));
      ptrs.push_back(d);
      dims.push_back(make_int4(ox, oy, oz, 0));
    }
    MMC_TRY(upload(c, &c->d_oct, ptrs));
    MMC_TRY(upload(c, &c->d_oct_dim, dims));
  }
  MMC_TRY(dalloc_t(c, &c->d_prop, (size_t)c->m_total));
  // shared memory: the largest need among the chains that fit in 200 KB
  size_t need = 0;
  for (const ChainDev &D : c->ch) {
    const size_t b = serial_smem_need(D);
    if (b <= 200 * 1024) need = std::max(need, b);
  }
  c->serial_smem = need;
  if (need > 0) CUDA_TRY(serial_set_smem_limit(need));
  c->serial_ready = true;
  return MMC_OK;
}

SerialLaunch serial_launch(mmc_ctx *c, unsigned off, unsigned key0, unsigned key1) {
  SerialLaunch P;
  P.chains = c->d_ch;
  P.st = c->d_st;
  P.m = c->d_m;
  P.heff = c->d_heff;
  P.tab = c->d_tab;
  P.ms = c->d_ms;
  P.oct = (const float *const *)c->d_oct;
  P.oct_dim = c->d_oct_dim;
  P.prop = c->d_prop;
  P.sweep_base = c->d_sweep_base;
  P.sweep_off = off;
  P.key0 = key0;
  P.key1 = key1;
  P.nchains = c->nchains;
  P.percell = c->any_percell;
  P.self = c->opt.demag_self != 0;
  P.smem = c->serial_smem;
  return P;
}

}  // namespace

// ===========================================================================
// C ABI
extern "C" {

mmc_status mmc_default_options(mmc_options *o) {
  if (!o) return fail(MMC_ERR_ARG, "null options");
  std::memset(o, 0, sizeof(*o));
  o->adapt = 1;
  o->theta0_deg = 30.0;
  o->sigma_cap = 0.03;
  o->hist_bins = 200;
  o->hist_max = 1.0;
  o->use_graphs = 1;
  o->stream_groups = 0;
  o->demag_self = 0;
  o->fft_variant = 0;
  o->demag_stripes = 1;
  o->sweep_tiles = 0;
  o->fuse_passes = 1;
  o->wait_polls = 0;
  o->wait_test = 0;
  return MMC_OK;
}

// checked builds: bad indices met by the contexts destroyed so far, and the
// site of the first of them
static std::atomic<long long> g_check_total{0};
static std::atomic<int> g_check_site{0};

void mmc_destroy(mmc_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (kChecked && c->d_check) {
    MmcCheck r;
    if (cudaMemcpy(&r, c->d_check, sizeof(r), cudaMemcpyDeviceToHost) == cudaSuccess && r.count) {
      int none = 0;
      g_check_site.compare_exchange_strong(none, r.site);
      g_check_total += (long long)r.count;
    }
  }
  for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (auto &g : c->cf) destroy_cufft_plans(g);
  for (auto &g : c->groups) {
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (void *p : c->allocs) cudaFree(p);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

mmc_status mmc_create(const mmc_chain_desc *chains, int nchains, const mmc_options *opt,
                      void *stream, mmc_ctx **out) {
  Trace trace("mmc_create");
  if (!out) return fail(MMC_ERR_ARG, "null output pointer");
  *out = nullptr;
  if (!chains || nchains < 1) return fail(MMC_ERR_ARG, "need at least one chain");
  mmc_options o;
  if (opt) o = *opt; else mmc_default_options(&o);
  if (o.hist_bins < 1 || o.hist_bins > kHistMax) return fail(MMC_ERR_ARG, "hist_bins must be in [1, 1024]");
  if (!(o.hist_max > 0)) return fail(MMC_ERR_ARG, "hist_max must be > 0");
  if (!(o.sigma_cap > 0 && o.sigma_cap < 1)) return fail(MMC_ERR_ARG, "sigma_cap must be in (0, 1)");
  if (!(o.theta0_deg >= 1 && o.theta0_deg <= 180)) return fail(MMC_ERR_ARG, "theta0_deg must be in [1, 180]");
  if (o.demag_stripes < 0 || o.demag_stripes > 64) return fail(MMC_ERR_ARG, "demag_stripes must be in [0, 64]");
  if (o.demag_fp64 < 0 || o.demag_fp64 > 2) return fail(MMC_ERR_ARG, "demag_fp64 must be 0, 1 or 2");
  if (o.chain_base < 0 || (long long)o.chain_base + nchains > 2147483647LL)
    return fail(MMC_ERR_ARG, "chain_base must be >= 0 with chain_base + nchains < 2^31");
  for (int i = 0; i < nchains; ++i) MMC_TRY(validate(chains[i], o, i));
  {
    bool any_pc = false, any_cubic = false;
    for (int i = 0; i < nchains; ++i) {
      any_pc |= has_percell(chains[i]);
      any_cubic |= chains[i].material.aniso_cubic != 0;
    }
    if (any_pc && any_cubic)
      return fail(MMC_ERR_UNSUPPORTED, "cubic anisotropy in a batch with per-cell material or temperature");
  }

  mmc_ctx *c = new mmc_ctx();
  c->nchains = nchains;
  c->opt = o;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) {
      delete c;
      return fail(MMC_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  CUDA_TRY_OR(demag_set_smem_limits());
  c->hc.resize(nchains);
  c->ch.resize(nchains);
  bool batch_percell = false;
  for (int i = 0; i < nchains; ++i) batch_percell |= has_percell(chains[i]);
  for (int i = 0; i < nchains; ++i) {
    build_chain(c->hc[i], c->ch[i], chains[i], o, i, batch_percell);
    c->any_demag |= (o.demag != 0);
    c->any_percell |= c->hc[i].percell;
    c->max_ncell = std::max(c->max_ncell, c->hc[i].ncell);
    c->max_slots = std::max(c->max_slots, c->hc[i].slots);
    c->all_flat = c->all_flat && chains[i].mesh.nz == 1;
  }
  // arenas
  long long moff = 0, toff = 0, msoff = 0, soff = 0;
  for (int i = 0; i < nchains; ++i) {
    ChainDev &D = c->ch[i];
    const long long S = c->hc[i].slots;
    D.m_off = moff;
    if (o.demag) D.h_off = moff;
    moff += 2 * S;
    if (c->hc[i].percell) {
      D.t_off = toff;
      toff += 6 * S;
      D.ms_off = msoff;
      msoff += 2 * S;
    }
    D.Px = D.Py = D.Pz = 1;
    if (o.demag) {
      // periodic demag axes whose extent is a power of two are transformed
      // circularly (length n); the others are zero padded to >= 2 n
      DemagPeriodic pd;
      {
        const mmc_mesh &ms = c->hc[i].mesh;
        const int ext[3] = {ms.nx, ms.ny, ms.nz};
        for (int a = 0; a < 3; ++a) {
          pd.n[a] = ext[a];
          pd.per[a] = ms.periodic[a] ? 1 : 0;
          pd.circ[a] = ms.demag_images > 0 && ms.periodic[a] && ext[a] >= kCircMin &&
                       (ext[a] & (ext[a] - 1)) == 0;
        }
        pd.images = ms.demag_images;
      }
      D.circ = (pd.circ[0] ? 1 : 0) | (pd.circ[1] ? 2 : 0) | (pd.circ[2] ? 4 : 0);
      D.Px = pd.circ[0] ? D.nx : pad_len(D.nx, true);
      D.Py = pd.circ[1] ? D.ny : pad_len(D.ny, true);
      D.Pz = pd.circ[2] ? D.nz : pad_len(D.nz, D.nz > 1);
      D.lx = ilog2(D.Px); D.ly = ilog2(D.Py); D.lz = ilog2(D.Pz);
      // spectrum row stride: a multiple of 8 and of the column-group width
      // 4096 / Py of the tiled 2D layout
      {
        const int g = std::max(8, D.Pz == 1 ? il_elements(false) / 3 / D.Py : 8);
        D.Sx = (D.Px / 2 + 1 + g - 1) / g * g;
      }
      D.s_off = soff;
      soff += 3LL * spectrum_rows(D) * D.Sx;
      int found = -1;
      for (size_t s = 0; s < c->specs.size(); ++s) {
        const SpecSet &ss = c->specs[s];
        if (ss.Px == D.Px && ss.Py == D.Py && ss.Pz == D.Pz && ss.h[0] == c->hc[i].h[0] &&
            ss.h[1] == c->hc[i].h[1] && ss.h[2] == c->hc[i].h[2] && ss.pd == pd)
          found = (int)s;
      }
      if (found < 0) {
        SpecSet ss;
        for (int a = 0; a < 3; ++a) ss.h[a] = c->hc[i].h[a];
        ss.Px = D.Px; ss.Py = D.Py; ss.Pz = D.Pz;
        ss.pd = pd;
        c->specs.push_back(ss);
        found = (int)c->specs.size() - 1;
      }
      D.spec = found;
    }
  }
  c->m_total = moff;
  c->tab_total = toff;
  c->ms_total = msoff;

  // initial state and per-cell tables, split layout
  {
    std::vector<float4> m((size_t)moff, make_float4(0, 0, 0, 0));
    std::vector<float4> tab((size_t)std::max(toff, 1LL), make_float4(0, 0, 0, 0));
    std::vector<float> ms((size_t)std::max(msoff, 1LL), 0.f), ms_lo(ms.size(), 0.f);
    std::vector<double> etab_all;
    for (int ci = 0; ci < nchains; ++ci) {
      const ChainDev &D = c->ch[ci];
      const ChainHost &H = c->hc[ci];
      const long long S = H.slots;
      for (int row = 0; row < D.nrows; ++row)
        for (int i = 0; i < D.nx; ++i) {
          const long long nat = i + (long long)D.nx * row;
          const long long si = split_index(D, i, row);
          const float g = H.grain.empty() ? 0.f : H.grain[(size_t)nat];
          m[(size_t)(D.m_off + si)] = make_float4(H.init_len[(size_t)nat], 0.f, 0.f, g);
        }
      if (H.percell) fill_percell_tables(H, D, tab.data() + D.t_off, ms.data() + D.ms_off, ms_lo.data() + D.ms_off);
    }
    MMC_TRY_OR(upload(c, &c->d_m, m));
    if (toff) MMC_TRY_OR(upload(c, &c->d_tab, tab));
    if (msoff) MMC_TRY_OR(upload(c, &c->d_ms, ms));
    if (msoff) MMC_TRY_OR(upload(c, &c->d_ms_lo, ms_lo));
    if (o.demag) MMC_TRY_OR(dalloc_t(c, &c->d_heff, (size_t)moff));
  }
  // tensor spectra and twiddles
  if (o.demag) {
    std::vector<void *> p32, p64, p32t, pff;
    for (auto &ss : c->specs) {
      std::vector<double> sp;
      demag_spectra(ss.h, ss.Px, ss.Py, ss.Pz, sp, ss.pd);
      if (o.demag_fp64 == 2) {
        // float-float copy: each FP64 value as its leading FP32 part and the rounded rest
        std::vector<float2> f(sp.size());
        for (size_t k = 0; k < sp.size(); ++k) {
          f[k].x = (float)sp[k];
          f[k].y = (float)(sp[k] - (double)f[k].x);
        }
        float2 *d = nullptr;
        MMC_TRY_OR(upload(c, &d, f));
        pff.push_back(d);
      }
      std::vector<float> spf(sp.begin(), sp.end());
      float *d32 = nullptr;
      double *d64 = nullptr;
      MMC_TRY_OR(upload(c, &d32, spf));
      MMC_TRY_OR(upload(c, &d64, sp));
      ss.d32 = d32;
      ss.d64 = d64;
      p32.push_back(d32);
      p64.push_back(d64);
      void *d32t = nullptr;
      if (ss.Px == 1024 && ss.Py == 1024 && ss.Pz == 1 && !ss.pd.circ[0] && !ss.pd.circ[1]) {
        // [comp][kyq][kx] -> [comp][kx][kyq] for the column blocks of the warp-transform path
        const size_t q = 513, tp = (size_t)kW32TensorPitch;
        std::vector<float> tr(4 * q * tp, 0.f);
        for (size_t cp = 0; cp < 4; ++cp)
          for (size_t ky = 0; ky < q; ++ky)
            for (size_t kx = 0; kx < q; ++kx) tr[(cp * q + kx) * tp + ky] = (float)sp[(cp * q + ky) * q + kx];
        float *dt = nullptr;
        MMC_TRY_OR(upload(c, &dt, tr));
        d32t = dt;
      }
      ss.d32t = d32t;
      p32t.push_back(d32t);
    }
    MMC_TRY_OR(upload(c, &c->d_nhat32, p32));
    MMC_TRY_OR(upload(c, &c->d_nhat64, p64));
    if (o.demag_fp64 == 2) {
      auto split = [](double v, float &hi, float &lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
      };
      MMC_TRY_OR(upload(c, &c->d_nhatff, pff));
      std::vector<float4> twf(kMaxFFT);
      for (int t = 0; t < kMaxFFT; ++t) {
        const double a = -2.0 * kPi * t / kMaxFFT;
        split(std::cos(a), twf[t].x, twf[t].y);
        split(std::sin(a), twf[t].z, twf[t].w);
      }
      float4 *d = nullptr;
      MMC_TRY_OR(upload(c, &d, twf));
      c->d_twff = d;
    }
    MMC_TRY_OR(upload(c, &c->d_nhat32t, p32t));
    {
      // 32 x 32 twiddles of the warp transforms: entry k1 * 32 + t = exp(-2 pi i t k1 / 1024)
      std::vector<float2> t1024(1024);
      for (int k1 = 0; k1 < 32; ++k1)
        for (int t = 0; t < 32; ++t) {
          const double a = -2.0 * kPi * (double)(t * k1) / 1024.0;
          t1024[(size_t)(k1 * 32 + t)] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
      float2 *d = nullptr;
      MMC_TRY_OR(upload(c, &d, t1024));
      c->d_tw1024 = d;
    }
    std::vector<float2> tw32(kMaxFFT);
    std::vector<double2> tw64(kMaxFFT);
    for (int t = 0; t < kMaxFFT; ++t) {
      const double a = -2.0 * kPi * t / kMaxFFT;
      tw64[t] = make_double2(std::cos(a), std::sin(a));
      tw32[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    float2 *t32 = nullptr;
    double2 *t64 = nullptr;
    MMC_TRY_OR(upload(c, &t32, tw32));
    MMC_TRY_OR(upload(c, &t64, tw64));
    c->d_tw32 = t32;
    c->d_tw64 = t64;
  }
  MMC_TRY_OR(upload(c, &c->d_ch, c->ch));
  {
    std::vector<ChainState> st((size_t)nchains);
    std::memset(st.data(), 0, st.size() * sizeof(ChainState));
    for (auto &s : st) {
      s.theta_deg = (float)o.theta0_deg;
      s.omc = (float)(1.0 - std::cos(o.theta0_deg * kPi / 180.0));
    }
    MMC_TRY_OR(upload(c, &c->d_st, st));
    MMC_TRY_OR(upload(c, &c->d_st_dbg, st));
    std::vector<unsigned> z(1, 0u);
    MMC_TRY_OR(upload(c, &c->d_sweep_base, z));
    MMC_TRY_OR(upload(c, &c->d_dbg_sweep, z));
  }
  // block tables
  {
    std::vector<int> bc;
    std::vector<long long> bf;
    for (int ci = 0; ci < nchains; ++ci) {
      bf.push_back((long long)bc.size());
      const long long nb = (c->hc[ci].slots + kSweepBlock - 1) / kSweepBlock;
      for (long long b = 0; b < nb; ++b) bc.push_back(ci);
    }
    bf.push_back((long long)bc.size());
    c->sw_first = bf;
    c->sw_blocks = (int)bc.size();
    MMC_TRY_OR(upload(c, &c->d_sw_chain, bc));
    MMC_TRY_OR(upload(c, &c->d_sw_first, bf));
    // one 8-byte descriptor per block (chain, block index within the chain):
    // a single load tells a sweep block where it works
    std::vector<int2> bd(bc.size());
    for (size_t b = 0; b < bc.size(); ++b) bd[b] = make_int2(bc[b], (int)((long long)b - bf[(size_t)bc[b]]));
    MMC_TRY_OR(upload(c, &c->d_sw_desc, bd));
    // bands of the banded pass: R rows of a chain with R hx <= 512 slots
    bool band = o.sweep_tiles != 0 && c->all_flat && !c->any_percell;
    for (int ci = 0; ci < nchains && band; ++ci) band = c->ch[ci].hx <= 512;
    if (band) {
      std::vector<int4> items;
      int own = 0, other = 0;
      for (int ci = 0; ci < nchains; ++ci) {
        const ChainDev &D = c->ch[ci];
        const int R = std::max(1, 512 / D.hx);
        c->item_first.push_back((int)items.size());
        for (int r0 = 0; r0 < D.ny; r0 += R) items.push_back(make_int4(ci, r0, std::min(R, D.ny - r0), 0));
        own = std::max(own, R * D.hx);
        other = std::max(other, (R + 2) * D.hx);
      }
      c->item_first.push_back((int)items.size());
      MMC_TRY_OR(upload(c, &c->d_items, items));
      c->stage_own = own;
      c->stage_other = other;
      const size_t bytes = band_smem_bytes(own, other);
      CUDA_TRY_OR(band_set_smem(bytes));
      int dev = 0, nsm = 1;
      CUDA_TRY_OR(cudaGetDevice(&dev));
      CUDA_TRY_OR(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      c->band_grid = band_blocks_per_sm(bytes) * nsm;
      c->band = true;
    }
    MMC_TRY_OR(dalloc_t(c, &c->d_err, 1));
    CUDA_TRY_OR(cudaMemset(c->d_err, 0, sizeof(int)));
    MMC_TRY_OR(dalloc_t(c, &c->d_check, 1));
    CUDA_TRY_OR(cudaMemset(c->d_check, 0, sizeof(MmcCheck)));
    std::vector<int> oc;
    std::vector<long long> of;
    for (int ci = 0; ci < nchains; ++ci) {
      of.push_back((long long)oc.size());
      const long long nb = (2 * c->hc[ci].slots + kReduceBlock * 4 - 1) / (kReduceBlock * 4);
      for (long long b = 0; b < nb; ++b) oc.push_back(ci);
    }
    of.push_back((long long)oc.size());
    c->obs_blocks = (int)oc.size();
    MMC_TRY_OR(upload(c, &c->d_obs_chain, oc));
    MMC_TRY_OR(upload(c, &c->d_obs_first, of));
    const long long eblocks = (2 * c->max_slots + kReduceBlock * 4 - 1) / (kReduceBlock * 4);
    MMC_TRY_OR(dalloc_t(c, &c->d_part, (size_t)8 * std::max<long long>(c->obs_blocks, eblocks)));
    const size_t hn = (size_t)nchains * (o.hist_bins + 1);
    MMC_TRY_OR(dalloc_t(c, &c->d_hist_acc, hn));
    MMC_TRY_OR(dalloc_t(c, &c->d_hist_cur, hn));
    CUDA_TRY_OR(cudaMemset(c->d_hist_acc, 0, hn * sizeof(unsigned long long)));
    MMC_TRY_OR(dalloc_t(c, &c->d_obs_out, (size_t)8 * nchains));
    MMC_TRY_OR(dalloc_t(c, &c->d_Hd, (size_t)3 * c->max_ncell));
    MMC_TRY_OR(dalloc_t(c, &c->d_eout, 8));
    MMC_TRY_OR(dalloc_t(c, &c->d_nat, (size_t)c->max_ncell));
    MMC_TRY_OR(dalloc_t(c, &c->d_dec, (size_t)c->max_ncell));
    MMC_TRY_OR(dalloc_t(c, &c->d_acc, (size_t)c->max_ncell));
  }
  if (o.demag) {
    std::vector<int> all(nchains);
    for (int i = 0; i < nchains; ++i) all[i] = i;
    MMC_TRY_OR(build_demag_plan(c, c->batch_plan, all, o.demag_fp64 != 0, false));
  }
  // autotuning: the FFT variant of the FP32 2D demag kernels and the number of
  // chain groups that iterate on concurrent streams, timed on this batch unless
  // the tuning cache holds picks for the same problem on this GPU model
  const bool want_fft = o.demag && !o.demag_cufft && !o.demag_fp64 && c->batch_plan.il2d && o.fft_variant == 0;
  const bool want_groups = o.stream_groups == 0 && nchains >= 2 && !o.demag_cufft;
  const std::string cpath = (want_fft || want_groups) ? tune_cache_path() : std::string();
  std::string tkey;
  int cached_fft = 0, cached_groups = 0;
  if (!cpath.empty()) {
    tkey = tune_key(c);
    c->tune_cached = tune_cache_read(cpath, tkey, cached_fft, cached_groups);
  }
  if (want_fft) {
    const auto usable = [&](int v) {
      return v >= 1 && v <= 4 && (v != 3 || c->batch_plan.small.ok) && (v != 4 || c->batch_plan.w32.ok);
    };
    int pick = 1;
    if (c->tune_cached && usable(cached_fft)) {
      pick = cached_fft;
    } else {
      // time the FP32 variants on this batch (a few updates each) and keep the fastest
      float best = 1e30f;
      cudaEvent_t e0, e1;
      CUDA_TRY_OR(cudaEventCreate(&e0));
      CUDA_TRY_OR(cudaEventCreate(&e1));
      for (int v = 1; v <= 4; ++v) {
        if (!usable(v)) continue;
        c->batch_plan.fft_variant = v;
        issue_demag(c);
        CUDA_TRY_OR(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < 5; ++r) issue_demag(c);
        CUDA_TRY_OR(cudaEventRecord(e1, c->stream));
        CUDA_TRY_OR(cudaEventSynchronize(e1));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        c->tune_ms[v - 1] = ms / 5.0;
        if (ms < best) { best = ms; pick = v; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      c->tune_cached = false;
    }
    c->batch_plan.fft_variant = pick;
    c->tuned_variant = pick;
  }
  int G = 1;
  if (o.stream_groups == 1 || nchains < 2 || o.demag_cufft) {
    G = 1;
  } else if (o.stream_groups > 1) {
    G = std::min(o.stream_groups, nchains);
  } else if (c->tune_cached && cached_groups >= 1 && (cached_fft == c->tuned_variant || !want_fft)) {
    G = std::min(cached_groups, nchains);
  } else {
    // time whole iterations with 1, 2 and 3 groups on a saved copy of the state
    // (the timing iterations are real moves; the state, the window counters and
    // the iteration counter are put back afterwards)
    void *save_m = nullptr, *save_st = nullptr;
    const size_t bm = (size_t)c->m_total * sizeof(float4), bs = (size_t)nchains * sizeof(ChainState);
    CUDA_TRY_OR(cudaMalloc(&save_m, bm));
    if (cudaMalloc(&save_st, bs) != cudaSuccess) {
      cudaFree(save_m);
      mmc_destroy(c);
      return fail(MMC_ERR_NOMEM, "cudaMalloc of the tuning copy failed");
    }
    unsigned save_base = 0;
    cudaMemcpyAsync(save_m, c->d_m, bm, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(save_st, c->d_st, bs, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(&save_base, c->d_sweep_base, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    mmc_status st = MMC_OK;
    for (int gcount = 1; gcount <= std::min(3, nchains) && st == MMC_OK; ++gcount) {
      st = make_groups(c, gcount);
      if (st != MMC_OK) break;
      issue_block(c, 5, 1u, 0u, 0, 0);
      cudaEventRecord(e0, c->stream);
      issue_block(c, 10, 1u, 0u, 0, 0);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      c->group_ms[gcount - 1] = ms / 10.0;
      if (ms < best) { best = ms; G = gcount; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(c->d_m, save_m, bm, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->d_st, save_st, bs, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->d_sweep_base, &save_base, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(save_m);
    cudaFree(save_st);
    if (st != MMC_OK) {
      mmc_destroy(c);
      return st;
    }
    CUDA_TRY_OR(cudaGetLastError());
    c->tune_cached = false;
  }
  if (want_groups) c->tuned_groups = G;
  MMC_TRY_OR(make_groups(c, G));
  if (!cpath.empty() && !c->tune_cached) tune_cache_write(cpath, tkey, c->tuned_variant, G);
  if (o.demag && o.demag_cufft) {
    // one batched cuFFT plan pair per padded size
    for (int i = 0; i < nchains; ++i) {
      const ChainDev &D = c->ch[i];
      CufftGroup *G = nullptr;
      for (auto &g : c->cf)
        if (g.Px == D.Px && g.Py == D.Py && g.Pz == D.Pz) G = &g;
      if (!G) {
        c->cf.emplace_back();
        G = &c->cf.back();
        G->Px = D.Px; G->Py = D.Py; G->Pz = D.Pz;
        G->fp64 = o.demag_fp64 != 0;
      }
      G->nchain += 1;
    }
    for (auto &G : c->cf) {
      std::vector<int> slots;
      for (int i = 0; i < nchains; ++i)
        if (c->ch[i].Px == G.Px && c->ch[i].Py == G.Py && c->ch[i].Pz == G.Pz) slots.push_back(i);
      MMC_TRY_OR(upload(c, &G.chain_of, slots));
      const size_t rs = G.fp64 ? 8 : 4;
      const long long P = (long long)G.Px * G.Py * G.Pz;
      const long long H = (long long)(G.Px / 2 + 1) * G.Py * G.Pz;
      MMC_TRY_OR(dalloc(c, &G.real, (size_t)G.nchain * 3 * P * rs));
      MMC_TRY_OR(dalloc(c, &G.cplx, (size_t)G.nchain * 3 * H * 2 * rs));
      if (make_cufft_plans(G) != cudaSuccess) {
        mmc_destroy(c);
        return fail(MMC_ERR_CUDA, "cufftPlanMany failed");
      }
    }
  }
  CUDA_TRY_OR(cudaDeviceSynchronize());
  *out = c;
  return MMC_OK;
}

mmc_status mmc_create_single(const mmc_mesh *mesh, const double cellsize[3], const mmc_material *mat,
                             double T, const double *T_cell, const mmc_options *opt, void *stream,
                             mmc_ctx **out) {
  if (!mesh || !cellsize || !mat) return fail(MMC_ERR_ARG, "null mesh, cell size or material");
  mmc_chain_desc d;
  std::memset(&d, 0, sizeof(d));
  d.mesh = *mesh;
  for (int a = 0; a < 3; ++a) d.cellsize[a] = cellsize[a];
  d.material = *mat;
  d.T = T;
  d.T_cell = T_cell;
  return mmc_create(&d, 1, opt, stream, out);
}

static mmc_status check_chain(mmc_ctx *c, int chain) {
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (chain < 0 || chain >= c->nchains) return fail(MMC_ERR_ARG, "chain index out of range");
  return MMC_OK;
}

mmc_status mmc_set_field(mmc_ctx *c, int chain, const double B[3]) {
  if (!c || !B) return fail(MMC_ERR_ARG, "null argument");
  if (chain >= c->nchains) return fail(MMC_ERR_ARG, "chain index out of range");
  for (int i = 0; i < c->nchains; ++i) {
    if (chain >= 0 && i != chain) continue;
    c->ch[i].Bx = (float)B[0];
    c->ch[i].By = (float)B[1];
    c->ch[i].Bz = (float)B[2];
    for (int a = 0; a < 3; ++a) c->hc[i].ecoef.B[a] = B[a];
    CUDA_TRY(cudaMemcpyAsync(c->d_ch + i, &c->ch[i], sizeof(ChainDev), cudaMemcpyHostToDevice, c->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->heff_stale = true;
  return MMC_OK;
}

mmc_status mmc_set_temperature(mmc_ctx *c, int chain, double T, const double *T_cell) {
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (chain >= c->nchains) return fail(MMC_ERR_ARG, "chain index out of range");
  if (!(T > 0)) return fail(MMC_ERR_ARG, "T must be > 0");
  if (T_cell && chain < 0) return fail(MMC_ERR_ARG, "per-cell temperatures need one chain");
  if (T_cell) {
    const ChainHost &H = c->hc[chain];
    if (!H.percell) return fail(MMC_ERR_UNSUPPORTED, "per-cell temperature on a chain created without per-cell tables");
    for (long long i = 0; i < H.ncell; ++i)
      if (!(T_cell[i] > 0)) return fail(MMC_ERR_ARG, "T_cell must be > 0");
  }
  for (int i = 0; i < c->nchains; ++i) {
    if (chain >= 0 && i != chain) continue;
    ChainHost &H = c->hc[i];
    ChainDev &D = c->ch[i];
    apply_temperature(H, D, c->opt, T, T_cell);
    if (H.percell) {
      std::vector<float4> tab((size_t)(6 * H.slots));
      std::vector<float> ms((size_t)(2 * H.slots)), ms_lo(ms.size());
      fill_percell_tables(H, D, tab.data(), ms.data(), ms_lo.data());
      CUDA_TRY(cudaMemcpyAsync(c->d_tab + D.t_off, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice,
                               c->stream));
      CUDA_TRY(cudaMemcpyAsync(c->d_ms + D.ms_off, ms.data(), ms.size() * sizeof(float), cudaMemcpyHostToDevice,
                               c->stream));
      CUDA_TRY(cudaMemcpyAsync(c->d_ms_lo + D.ms_off, ms_lo.data(), ms_lo.size() * sizeof(float),
                               cudaMemcpyHostToDevice, c->stream));
      CUDA_TRY(cudaStreamSynchronize(c->stream));   // the host vectors go out of scope
    }
    CUDA_TRY(cudaMemcpyAsync(c->d_ch + i, &D, sizeof(ChainDev), cudaMemcpyHostToDevice, c->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->heff_stale = true;
  return MMC_OK;
}

mmc_status mmc_demag_update(mmc_ctx *c) {
  Trace trace("mmc_demag_update");
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (!c->any_demag) return MMC_OK;
  issue_demag(c);
  MMC_TRY(check_launch());
  c->heff_stale = false;
  return MMC_OK;
}

mmc_status mmc_set_m(mmc_ctx *c, int chain, const float *src, int is_device) {
  MMC_TRY(check_chain(c, chain));
  if (!src) return fail(MMC_ERR_ARG, "null source");
  const long long n = c->hc[chain].ncell;
  if (!c->d_flag) MMC_TRY(dalloc_t(c, &c->d_flag, 1));
  CUDA_TRY(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->d_nat, src, (size_t)n * sizeof(float4),
                           is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  Launch L = c->L();
  // the copy is checked on the device before the state is touched; the wait
  // below also ends the use of the caller's buffer
  launch_check_finite(L, c->d_nat, n, c->d_flag);
  MMC_TRY(check_launch());
  int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (bad) return fail(MMC_ERR_NONFINITE, "non-finite value in m");
  launch_pack(L, c->d_ch, chain, c->hc[chain].slots, c->d_m, c->d_nat, 1);
  MMC_TRY(check_launch());
  c->heff_stale = true;
  c->obs_fresh = false;
  return MMC_OK;
}

mmc_status mmc_get_m(mmc_ctx *c, int chain, float *dst, int is_device) {
  MMC_TRY(check_chain(c, chain));
  if (!dst) return fail(MMC_ERR_ARG, "null destination");
  const long long n = c->hc[chain].ncell;
  Launch L = c->L();
  launch_pack(L, c->d_ch, chain, c->hc[chain].slots, c->d_m, c->d_nat, 0);
  MMC_TRY(check_launch());
  CUDA_TRY(cudaMemcpyAsync(dst, c->d_nat, (size_t)n * sizeof(float4),
                           is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MMC_OK;
}

// the natural-order buffer of the whole batch, allocated on first use
static mmc_status nat_all(mmc_ctx *c, long long *n) {
  long long tot = 0;
  for (int k = 0; k < c->nchains; ++k) tot += c->hc[k].ncell;
  if (!c->d_nat_all) MMC_TRY(dalloc_t(c, &c->d_nat_all, (size_t)tot));
  *n = tot;
  return MMC_OK;
}

mmc_status mmc_set_m_all(mmc_ctx *c, const float *src, int is_device) {
  Trace trace("mmc_set_m_all");
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (!src) return fail(MMC_ERR_ARG, "null source");
  long long n = 0;
  MMC_TRY(nat_all(c, &n));
  if (!c->d_flag) MMC_TRY(dalloc_t(c, &c->d_flag, 1));
  CUDA_TRY(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->d_nat_all, src, (size_t)n * sizeof(float4),
                           is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  Launch L = c->L();
  launch_check_finite(L, c->d_nat_all, n, c->d_flag);
  MMC_TRY(check_launch());
  int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (bad) return fail(MMC_ERR_NONFINITE, "non-finite value in m");
  long long off = 0;
  for (int k = 0; k < c->nchains; ++k) {
    launch_pack(L, c->d_ch, k, c->hc[k].slots, c->d_m, c->d_nat_all + off, 1);
    off += c->hc[k].ncell;
  }
  MMC_TRY(check_launch());
  c->heff_stale = true;
  c->obs_fresh = false;
  return MMC_OK;
}

mmc_status mmc_get_m_all(mmc_ctx *c, float *dst, int is_device) {
  Trace trace("mmc_get_m_all");
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (!dst) return fail(MMC_ERR_ARG, "null destination");
  long long n = 0;
  MMC_TRY(nat_all(c, &n));
  Launch L = c->L();
  long long off = 0;
  for (int k = 0; k < c->nchains; ++k) {
    launch_pack(L, c->d_ch, k, c->hc[k].slots, c->d_m, c->d_nat_all + off, 0);
    off += c->hc[k].ncell;
  }
  MMC_TRY(check_launch());
  CUDA_TRY(cudaMemcpyAsync(dst, c->d_nat_all, (size_t)n * sizeof(float4),
                           is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MMC_OK;
}

mmc_status mmc_init_random(mmc_ctx *c, uint64_t seed, double len) {
  if (!c) return fail(MMC_ERR_ARG, "null context");
  Launch L = c->L();
  float *d_len = nullptr;
  for (int ci = 0; ci < c->nchains; ++ci) {
    const ChainHost &H = c->hc[ci];
    const float *lp = nullptr;
    float lu = (float)len;
    if (!(len > 0)) {
      if (H.percell) {
        if (!d_len) MMC_TRY(dalloc_t(c, &d_len, (size_t)c->max_ncell));
        CUDA_TRY(cudaMemcpyAsync(d_len, H.init_len.data(), (size_t)H.ncell * sizeof(float),
                                 cudaMemcpyHostToDevice, c->stream));
        lp = d_len;
      } else {
        lu = H.init_len[0];
      }
    }
    launch_init_random(L, c->d_ch, ci, H.slots, c->d_m, (unsigned)(seed & 0xffffffffu),
                       (unsigned)(seed >> 32), lp, lu);
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  MMC_TRY(check_launch());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->heff_stale = true;
  c->obs_fresh = false;
  return MMC_OK;
}

mmc_status mmc_sweep(mmc_ctx *c, int64_t n, uint64_t seed) {
  Trace trace("mmc_sweep");
  MMC_TRY(sweep_impl(c, n, seed, 0));
  return MMC_OK;
}

mmc_status mmc_sweep_sampled(mmc_ctx *c, int64_t n, uint64_t seed, int sample_every) {
  Trace trace("mmc_sweep_sampled");
  if (sample_every < 1) return fail(MMC_ERR_ARG, "sample_every must be >= 1");
  MMC_TRY(sweep_impl(c, n, seed, sample_every));
  return MMC_OK;
}

mmc_status mmc_sweep_serial(mmc_ctx *c, int64_t n, uint64_t seed) {
  Trace trace("mmc_sweep_serial");
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (n < 0) return fail(MMC_ERR_ARG, "negative sweep count");
  MMC_TRY(serial_prepare(c));
  const unsigned key0 = (unsigned)(seed & 0xffffffffu), key1 = (unsigned)(seed >> 32);
  Launch L = c->L();
  while (n > 0) {
    const int k = (int)std::min<int64_t>(n, 100 - (int64_t)(c->host_sweep % 100));
    for (int off = 0; off < k; ++off) {
      if (c->any_demag) issue_demag(c);
      launch_serial_sweep(L, serial_launch(c, (unsigned)off, key0, key1));
    }
    const int adapt_now = ((c->host_sweep + k) % 100 == 0) ? 1 : 0;
    launch_advance(L, c->d_st, c->nchains, (unsigned)k, c->d_sweep_base, adapt_now, c->opt.adapt, 1.f, 180.f);
    MMC_TRY(check_launch());
    c->host_sweep += (uint64_t)k;
    n -= k;
  }
  c->heff_stale = true;
  c->obs_fresh = false;
  return MMC_OK;
}

mmc_status mmc_pass_debug(mmc_ctx *c, int chain, int color, uint32_t sweep, uint64_t seed,
                          double theta_deg, float *dec, int8_t *acc) {
  MMC_TRY(check_chain(c, chain));
  if (color != 0 && color != 1) return fail(MMC_ERR_ARG, "color must be 0 or 1");
  if (!(theta_deg >= 0 && theta_deg <= 180)) return fail(MMC_ERR_ARG, "theta_deg must be in [0, 180]");
  const long long n = c->hc[chain].ncell;
  if (c->any_demag && c->heff_stale) MMC_TRY(mmc_demag_update(c));
  CUDA_TRY(cudaMemcpyAsync(c->d_dbg_sweep, &sweep, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaMemsetAsync(c->d_dec, 0, (size_t)n * sizeof(float), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->d_acc, 0xff, (size_t)n, c->stream));
  SweepLaunch P = sweep_launch(c, color, 0u, (unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32));
  P.st = c->d_st_dbg;
  P.sweep_base = c->d_dbg_sweep;
  P.blk_base = (int)c->sw_first[chain];
  P.nblocks = (int)(c->sw_first[chain + 1] - c->sw_first[chain]);
  if (c->band) {
    P.i0 = c->item_first[(size_t)chain];
    P.i1 = c->item_first[(size_t)chain + 1];
  }
  P.omc_override = (float)(1.0 - std::cos(theta_deg * kPi / 180.0));
  P.dec_dbg = c->d_dec;
  P.acc_dbg = c->d_acc;
  Launch L = c->L();
  launch_sweep_pass(L, P);
  MMC_TRY(check_launch());
  c->obs_fresh = false;                 // accepted moves changed the state
  c->heff_stale = true;
  if (dec) CUDA_TRY(cudaMemcpyAsync(dec, c->d_dec, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (acc) CUDA_TRY(cudaMemcpyAsync(acc, c->d_acc, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MMC_OK;
}

// the error word of the kernels' bounded waits: a wait that gave up since the
// last check makes this call fail with MMC_ERR_TIMEOUT (and clears the word)
static mmc_status take_device_error(mmc_ctx *c) {
  if (!c->d_err) return MMC_OK;
  int e = 0;
  CUDA_TRY(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (e == 0) return MMC_OK;
  CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return fail(MMC_ERR_TIMEOUT, "a band of the sublattice pass gave up waiting for its copies; the bands that "
                               "gave up were not updated");
}

mmc_status mmc_observables(mmc_ctx *c, int chain, mmc_obs *out, int reset) {
  Trace trace("mmc_observables");
  MMC_TRY(check_chain(c, chain));
  if (!out) return fail(MMC_ERR_ARG, "null output");
  MMC_TRY(take_device_error(c));
  ChainState s;
  CUDA_TRY(cudaMemcpyAsync(&s, c->d_st + chain, sizeof(ChainState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const int nb = c->opt.hist_bins + 1;
  std::vector<unsigned long long> h((size_t)nb, 0);
  if (s.nsnap == 0) {
    if (!c->obs_fresh) {   // one reduction serves every chain until the state changes
      CUDA_TRY(cudaMemsetAsync(c->d_hist_cur, 0, (size_t)c->nchains * nb * sizeof(unsigned long long), c->stream));
      Launch L = c->L();
      launch_obs(L, obs_launch(c, 0));
      MMC_TRY(check_launch());
      c->obs_fresh = true;
    }
    double o[8];
    CUDA_TRY(cudaMemcpyAsync(o, c->d_obs_out + 8 * chain, sizeof(o), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(h.data(), c->d_hist_cur + (size_t)chain * nb, nb * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    const double nv = o[6] > 0 ? o[6] : 1.0;
    for (int a = 0; a < 3; ++a) out->mean_m[a] = o[a] / nv;
    out->mean_len = o[3] / nv;
    out->mean_len2 = o[4] / nv;
    out->nonfinite = (int64_t)o[5];
    out->nsnap = 0;
  } else {
    CUDA_TRY(cudaMemcpyAsync(h.data(), c->d_hist_acc + (size_t)chain * nb, nb * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    const double ns = s.nsamples > 0 ? (double)s.nsamples : 1.0;
    for (int a = 0; a < 3; ++a) out->mean_m[a] = s.sum_m[a] / ns;
    out->mean_len = s.sum_len / ns;
    out->mean_len2 = s.sum_len2 / ns;
    out->nonfinite = (int64_t)s.nonfinite;
    out->nsnap = (int64_t)s.nsnap;
  }
  if (out->hist)
    for (int b = 0; b < nb; ++b) out->hist[b] = (int64_t)h[(size_t)b];
  out->acc_rate = s.last_att > 0 ? (double)s.last_acc / (double)s.last_att : 0.0;
  out->theta_deg = s.theta_deg;
  out->sweeps = (int64_t)c->host_sweep;
  if (reset) {
    ChainState z = s;
    z.sum_m[0] = z.sum_m[1] = z.sum_m[2] = 0;
    z.sum_len = z.sum_len2 = 0;
    z.nsamples = z.nsnap = z.nonfinite = 0;
    CUDA_TRY(cudaMemcpyAsync(c->d_st + chain, &z, sizeof(ChainState), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_hist_acc + (size_t)chain * nb, 0, nb * sizeof(unsigned long long), c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  return MMC_OK;
}

mmc_status mmc_observables_all(mmc_ctx *c, mmc_obs *out, int reset) {
  Trace trace("mmc_observables_all");
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (!out) return fail(MMC_ERR_ARG, "null output");
  const int nc = c->nchains, nb = c->opt.hist_bins + 1;
  // the current-state reduction of every chain (cheap next to a sweep block),
  // then everything back in one round trip
  if (!c->obs_fresh) {
    CUDA_TRY(cudaMemsetAsync(c->d_hist_cur, 0, (size_t)nc * nb * sizeof(unsigned long long), c->stream));
    Launch L = c->L();
    launch_obs(L, obs_launch(c, 0));
    MMC_TRY(check_launch());
    c->obs_fresh = true;
  }
  std::vector<ChainState> st((size_t)nc);
  std::vector<double> o((size_t)8 * nc);
  std::vector<unsigned long long> hc((size_t)nc * nb), ha((size_t)nc * nb);
  int err = 0;
  if (c->d_err) CUDA_TRY(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(st.data(), c->d_st, st.size() * sizeof(ChainState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(o.data(), c->d_obs_out, o.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(hc.data(), c->d_hist_cur, hc.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaMemcpyAsync(ha.data(), c->d_hist_acc, ha.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (err) {
    CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return fail(MMC_ERR_TIMEOUT, "a band of the sublattice pass gave up waiting for its copies; the bands that "
                                 "gave up were not updated");
  }
  for (int k = 0; k < nc; ++k) {
    const ChainState &s = st[(size_t)k];
    mmc_obs &r = out[k];
    const unsigned long long *h = (s.nsnap == 0 ? hc.data() : ha.data()) + (size_t)k * nb;
    if (s.nsnap == 0) {
      const double *ok = o.data() + 8 * k;
      const double nv = ok[6] > 0 ? ok[6] : 1.0;
      for (int a = 0; a < 3; ++a) r.mean_m[a] = ok[a] / nv;
      r.mean_len = ok[3] / nv;
      r.mean_len2 = ok[4] / nv;
      r.nonfinite = (int64_t)ok[5];
      r.nsnap = 0;
    } else {
      const double ns = s.nsamples > 0 ? (double)s.nsamples : 1.0;
      for (int a = 0; a < 3; ++a) r.mean_m[a] = s.sum_m[a] / ns;
      r.mean_len = s.sum_len / ns;
      r.mean_len2 = s.sum_len2 / ns;
      r.nonfinite = (int64_t)s.nonfinite;
      r.nsnap = (int64_t)s.nsnap;
    }
    if (r.hist)
      for (int b = 0; b < nb; ++b) r.hist[b] = (int64_t)h[b];
    r.acc_rate = s.last_att > 0 ? (double)s.last_acc / (double)s.last_att : 0.0;
    r.theta_deg = s.theta_deg;
    r.sweeps = (int64_t)c->host_sweep;
  }
  if (reset) {
    for (auto &z : st) {
      z.sum_m[0] = z.sum_m[1] = z.sum_m[2] = 0;
      z.sum_len = z.sum_len2 = 0;
      z.nsamples = z.nsnap = z.nonfinite = 0;
    }
    CUDA_TRY(cudaMemcpyAsync(c->d_st, st.data(), st.size() * sizeof(ChainState), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->d_hist_acc, 0, (size_t)nc * nb * sizeof(unsigned long long), c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  return MMC_OK;
}

static mmc_status demag64_chain(mmc_ctx *c, int chain) {
  DemagPlan *P = nullptr;
  MMC_TRY(single_plan(c, chain, true, &P));
  Launch L = c->L();
  launch_demag(L, make_demag_launch(c, *P, nullptr, c->d_Hd, 0), true);
  return check_launch();
}

mmc_status mmc_angle_hist(mmc_ctx *c, int chain, int bins, double theta_lo, double theta_hi, int64_t *hist,
                          double mean_dir[3]) {
  MMC_TRY(check_chain(c, chain));
  if (!hist) return fail(MMC_ERR_ARG, "null histogram");
  if (bins < 1 || bins > kHistMax) return fail(MMC_ERR_ARG, "bins must be in [1, 1024]");
  if (!(theta_hi > theta_lo)) return fail(MMC_ERR_ARG, "theta_hi must exceed theta_lo");
  Launch L = c->L();
  // the mean direction from the current-state reduction (shared with mmc_observables)
  if (!c->obs_fresh) {
    const int nb = c->opt.hist_bins + 1;
    CUDA_TRY(cudaMemsetAsync(c->d_hist_cur, 0, (size_t)c->nchains * nb * sizeof(unsigned long long), c->stream));
    launch_obs(L, obs_launch(c, 0));
    MMC_TRY(check_launch());
    c->obs_fresh = true;
  }
  double o[8];
  CUDA_TRY(cudaMemcpyAsync(o, c->d_obs_out + 8 * chain, sizeof(o), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  double n[3] = {o[0], o[1], o[2]};
  const double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (l > 0) for (int a = 0; a < 3; ++a) n[a] /= l;
  else { n[0] = 0; n[1] = 0; n[2] = 1; }
  if (mean_dir) for (int a = 0; a < 3; ++a) mean_dir[a] = n[a];
  if (!c->d_ang) MMC_TRY(dalloc_t(c, &c->d_ang, (size_t)kHistMax + 1));
  unsigned long long *d_h = c->d_ang;
  CUDA_TRY(cudaMemsetAsync(d_h, 0, ((size_t)bins + 1) * sizeof(unsigned long long), c->stream));
  launch_angle_hist(L, c->d_ch, chain, c->hc[chain].slots, c->d_m, n, theta_lo, theta_hi, bins, d_h);
  MMC_TRY(check_launch());
  std::vector<unsigned long long> h((size_t)bins + 1);
  CUDA_TRY(cudaMemcpyAsync(h.data(), d_h, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int b = 0; b <= bins; ++b) hist[b] = (int64_t)h[(size_t)b];
  return MMC_OK;
}

mmc_status mmc_trial_terms(mmc_ctx *c, int chain, uint32_t sweep, uint64_t seed, double theta_deg,
                           double out[6]) {
  Trace trace("mmc_trial_terms");
  MMC_TRY(check_chain(c, chain));
  if (!out) return fail(MMC_ERR_ARG, "null output");
  if (!(theta_deg <= 180)) return fail(MMC_ERR_ARG, "theta_deg must be <= 180 (negative: the chain's angle)");
  if (c->any_demag && c->heff_stale) MMC_TRY(mmc_demag_update(c));
  const long long slots = c->hc[chain].slots;       // per colour
  const int nb = trial_terms_blocks(slots);
  if (!c->d_terms) MMC_TRY(dalloc_t(c, &c->d_terms, (size_t)6 * (trial_terms_blocks(c->max_slots) + 1)));
  const float omc = theta_deg >= 0 ? (float)(1.0 - std::cos(theta_deg * kPi / 180.0)) : -1.f;
  Launch L = c->L();
  launch_trial_terms(L, c->d_ch, c->d_st, chain, slots, c->ch[chain].t_off >= 0, c->d_m, c->d_heff, c->d_tab,
                     sweep, (unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32), omc, c->d_terms,
                     c->d_terms + 6 * (size_t)nb);
  MMC_TRY(check_launch());
  double sums[6];
  CUDA_TRY(cudaMemcpyAsync(sums, c->d_terms + 6 * (size_t)nb, sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const double n = (double)c->hc[chain].ncell;
  for (int k = 0; k < 6; ++k) out[k] = sums[k] / n;
  return MMC_OK;
}

mmc_status mmc_demag_field(mmc_ctx *c, int chain, double *H) {
  MMC_TRY(check_chain(c, chain));
  if (!H) return fail(MMC_ERR_ARG, "null output");
  const long long n = c->hc[chain].ncell;
  if (!c->any_demag) {
    std::memset(H, 0, (size_t)n * 3 * sizeof(double));
    return MMC_OK;
  }
  MMC_TRY(demag64_chain(c, chain));
  CUDA_TRY(cudaMemcpyAsync(H, c->d_Hd, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MMC_OK;
}

mmc_status mmc_sweep_field(mmc_ctx *c, int chain, double *H) {
  Trace trace("mmc_sweep_field");
  MMC_TRY(check_chain(c, chain));
  if (!H) return fail(MMC_ERR_ARG, "null output");
  const long long n = c->hc[chain].ncell;
  if (!c->any_demag) {
    std::memset(H, 0, (size_t)n * 3 * sizeof(double));
    return MMC_OK;
  }
  if (!c->cf.empty()) return fail(MMC_ERR_UNSUPPORTED, "the cuFFT comparison path does not report its field");
  // the batch plan with the kernels and precision the sweep uses; the chain's
  // field is also written out in natural order (h_eff gets the values the next
  // iteration would compute anyway)
  DemagLaunch D = make_demag_launch(c, c->batch_plan, c->d_heff, c->d_Hd, chain);
  launch_demag(c->L(), D, c->batch_plan.fp64);
  MMC_TRY(check_launch());
  CUDA_TRY(cudaMemcpyAsync(H, c->d_Hd, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MMC_OK;
}

mmc_status mmc_energy(mmc_ctx *c, int chain, double out[7]) {
  Trace trace("mmc_energy");
  MMC_TRY(check_chain(c, chain));
  if (!out) return fail(MMC_ERR_ARG, "null output");
  const ChainHost &H = c->hc[chain];
  if (c->any_demag) MMC_TRY(demag64_chain(c, chain));
  double *etab = nullptr;
  if (H.percell) {
    if (!c->d_etab) MMC_TRY(dalloc_t(c, &c->d_etab, (size_t)10 * c->max_ncell));
    CUDA_TRY(cudaMemcpyAsync(c->d_etab, H.etab.data(), H.etab.size() * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream));
    etab = c->d_etab;
  }
  Launch L = c->L();
  launch_energy(L, c->d_ch, chain, H.slots, c->d_m, etab, c->any_demag ? c->d_Hd : nullptr, H.ecoef, c->d_part,
                c->d_eout);
  MMC_TRY(check_launch());
  CUDA_TRY(cudaMemcpyAsync(out, c->d_eout, 7 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MMC_OK;
}

mmc_status mmc_tables(mmc_ctx *c, int chain, double *me, double *chi, double *sigma) {
  MMC_TRY(check_chain(c, chain));
  const ChainHost &H = c->hc[chain];
  for (long long i = 0; i < H.ncell; ++i) {
    const size_t k = H.percell ? (size_t)i : 0;
    if (me) me[i] = H.me[k];
    if (chi) chi[i] = H.chi[k];
    if (sigma) sigma[i] = H.sigma[k];
  }
  return MMC_OK;
}

mmc_status mmc_energy_grad(mmc_ctx *c, int chain, const void *m, int fp64, const double params[5],
                           double E[7], void *dEdm, double dEdp[5]) {
  Trace trace("mmc_energy_grad");
  MMC_TRY(check_chain(c, chain));
  if (!m || !E) return fail(MMC_ERR_ARG, "null m or E");
  const ChainHost &H = c->hc[chain];
  if (H.percell) return fail(MMC_ERR_UNSUPPORTED, "energy gradient of a chain with per-cell material");
  const bool f64 = fp64 != 0;
  double Ms0 = H.Ms0, A0 = H.ecoef.cex[0] * H.h[0] * H.h[0] / H.V, D0 = H.ecoef.cdmi[0] * H.h[0] / H.V;
  double Ku = H.K1, chi = H.chi[0];
  if (params) {
    Ms0 = params[0]; A0 = params[1]; D0 = params[2]; Ku = params[3]; chi = params[4];
    if (!(Ms0 > 0) || !(chi > 0)) return fail(MMC_ERR_ARG, "params: Ms0 and chi must be > 0");
  }
  GradCoef G;
  std::memset(&G, 0, sizeof(G));
  for (int a = 0; a < 3; ++a) {
    G.vh2[a] = H.V / (H.h[a] * H.h[a]);
    G.cex[a] = A0 * G.vh2[a];
  }
  for (int a = 0; a < 2; ++a) {
    G.vh[a] = H.V / H.h[a];
    G.cdmi[a] = D0 * G.vh[a];
  }
  const double me = H.me[0];
  const int l1 = H.cubic ? 10 : 3, l2 = H.cubic ? 21 : 10;
  G.Kscale = std::pow(me, l1);
  G.K1T = Ku * G.Kscale;
  G.K2T = H.K2 * std::pow(me, l2);
  for (int a = 0; a < 3; ++a) { G.e[a] = H.ecoef.e[a]; G.B[a] = H.ecoef.B[a]; }
  G.V = H.V;
  G.Ms0 = Ms0;
  G.cubic = H.cubic;
  G.anis = (Ku != 0.0 || H.K2 != 0.0) ? 1 : 0;
  G.dmi = 1;
  // longitudinal coefficients from Eq. 7 with the given chi
  {
    const double T = H.T, Tc = H.Tc;
    const double Tg = std::fabs(T - Tc) < 1e-3 ? (T < Tc ? Tc - 1e-3 : Tc + 1e-3) : T;
    if (Tg < Tc) {
      G.c2 = 0.0;
      G.c4 = H.V * Ms0 / (8.0 * chi * me * me);
      G.me2 = me * me;
    } else {
      G.c2 = H.V * Ms0 / (2.0 * chi);
      G.c4 = G.c2 * 3.0 * Tc / (10.0 * (Tg - Tc));
      G.me2 = 0.0;
    }
  }
  const double *Hd = nullptr;
  if (c->any_demag) {
    DemagPlan *P = nullptr;
    MMC_TRY(single_plan(c, chain, f64, &P));
    DemagLaunch D = make_demag_launch(c, *P, nullptr, c->d_Hd, 0);
    D.m_nat = m;
    D.Ms_override = Ms0;
    launch_demag(c->L(), D, f64);
    Hd = c->d_Hd;
  }
  if (!c->d_g8) MMC_TRY(dalloc_t(c, &c->d_g8, 8));
  launch_energy_grad(c->L(), c->d_ch, chain, H.ncell, m, f64, Hd, G, dEdm, c->d_part, c->d_g8);
  MMC_TRY(check_launch());
  double o[8];
  CUDA_TRY(cudaMemcpyAsync(o, c->d_g8, sizeof(o), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  // o = {ex_unit, dmi_unit, an, an1_unit, zee, long, demag}
  E[1] = A0 * o[0];
  E[2] = D0 * o[1];
  E[3] = o[2];
  E[4] = o[4];
  E[5] = o[5];
  E[6] = o[6];
  E[0] = E[1] + E[2] + E[3] + E[4] + E[5] + E[6];
  if (dEdp) {
    dEdp[0] = (E[5] + E[4] + 2.0 * E[6]) / Ms0;
    dEdp[1] = o[0];
    dEdp[2] = o[1];
    dEdp[3] = o[3];
    dEdp[4] = -E[5] / chi;
  }
  return MMC_OK;
}

mmc_status mmc_minimize(mmc_ctx *c, int chain, int64_t maxit, double tol, int64_t *iters, double *torque,
                        double E[7]) {
  Trace trace("mmc_minimize");
  MMC_TRY(check_chain(c, chain));
  if (!(tol > 0) || maxit < 0) return fail(MMC_ERR_ARG, "tol must be > 0 and maxit >= 0");
  const ChainHost &H = c->hc[chain];
  if (H.percell) return fail(MMC_ERR_UNSUPPORTED, "steepest descent of a chain with per-cell material");
  if (!(H.me[0] > 0)) return fail(MMC_ERR_ARG, "steepest descent needs T < Tc (m_e > 0)");
  const long long n = H.ncell;
  const double me = H.me[0];
  if (!c->d_sd) {
    MMC_TRY(dalloc_t(c, &c->d_sd, (size_t)18 * c->max_ncell));
    MMC_TRY(dalloc_t(c, &c->d_sd_part, (size_t)5 * sd_blocks(c->max_ncell)));
    MMC_TRY(dalloc_t(c, &c->d_sd_out, 8));
  }
  const size_t v3 = (size_t)3 * c->max_ncell;
  double *u = c->d_sd, *m = u + v3, *up = m + v3, *gp = up + v3, *G = gp + v3, *g = G + v3;
  Launch L = c->L();
  CUDA_TRY(cudaMemsetAsync(up, 0, 2 * v3 * sizeof(double), c->stream));
  launch_sd_init(L, c->d_ch, chain, n, c->d_m, me, u, m);
  MMC_TRY(check_launch());
  double tau = 0.0, tmax = 0.0, e7[7] = {0, 0, 0, 0, 0, 0, 0};
  int64_t it = 0;
  for (;;) {
    MMC_TRY(mmc_energy_grad(c, chain, m, 1, nullptr, e7, G, nullptr));
    launch_sd_dir(L, n, me, u, G, g, up, gp, c->d_sd_part, c->d_sd_out);
    MMC_TRY(check_launch());
    double o[5];
    CUDA_TRY(cudaMemcpyAsync(o, c->d_sd_out, sizeof(o), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    tmax = o[4];
    if (!(tmax >= tol) || it >= maxit) break;        // converged (or NaN torque), or out of steps
    if (it == 0) tau = o[3] > 0 ? 0.01 / std::sqrt(o[3]) : 0.0;
    else if (o[1] > 0) tau = (it & 1) ? o[0] / o[1] : o[1] / o[2];
    launch_sd_step(L, n, me, tau, u, g, up, gp, m);
    ++it;
  }
  launch_sd_store(L, c->d_ch, chain, n, m, c->d_m);
  MMC_TRY(check_launch());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->heff_stale = true;
  c->obs_fresh = false;
  if (iters) *iters = it;
  if (torque) *torque = tmax;
  if (E) for (int k = 0; k < 7; ++k) E[k] = e7[k];
  if (!(tmax == tmax)) return fail(MMC_ERR_NONFINITE, "steepest descent produced a non-finite torque");
  return MMC_OK;
}

mmc_status mmc_phase_times(mmc_ctx *c, int64_t n, uint64_t seed, double ms[8], int64_t count[8]) {
  if (!c || !ms || !count) return fail(MMC_ERR_ARG, "null argument");
  if (n < 0) return fail(MMC_ERR_ARG, "negative sweep count");
  for (int k = 0; k < 8; ++k) { ms[k] = 0; count[k] = 0; }
  const unsigned key0 = (unsigned)(seed & 0xffffffffu), key1 = (unsigned)(seed >> 32);
  PhaseTimer pt;
  mmc_status st = MMC_OK;
  while (n > 0 && st == MMC_OK) {
    const int k = (int)std::min<int64_t>(n, 100 - (int64_t)(c->host_sweep % 100));
    pt.used = 0;
    pt.marks.clear();
    issue_block(c, k, key0, key1, 0, c->host_sweep, &pt);
    st = check_launch();
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { st = fail(MMC_ERR_CUDA, cudaGetErrorString(e)); break; }
    for (auto &mk : pt.marks) {
      float t = 0;
      cudaEventElapsedTime(&t, pt.pool[mk.second.first], pt.pool[mk.second.second]);
      ms[mk.first] += t;
      count[mk.first] += 1;
    }
    c->host_sweep += (uint64_t)k;
    n -= k;
  }
  for (auto e : pt.pool) cudaEventDestroy(e);
  c->heff_stale = true;
  c->obs_fresh = false;
  return st;
}

int64_t mmc_kernel_launches(const mmc_ctx *c) { return c ? c->launches : 0; }

mmc_status mmc_tuning(const mmc_ctx *c, int *fft_variant, int *stream_groups, int *from_cache, double ms[7]) {
  if (!c) return fail(MMC_ERR_ARG, "null context");
  if (fft_variant) *fft_variant = c->batch_plan.ready && c->batch_plan.il2d ? c->batch_plan.fft_variant : 0;
  if (stream_groups) *stream_groups = c->groups.empty() ? 1 : (int)c->groups.size();
  if (from_cache) *from_cache = c->tune_cached ? 1 : 0;
  if (ms) {
    for (int k = 0; k < 4; ++k) ms[k] = c->tune_ms[k];
    for (int k = 0; k < 3; ++k) ms[4 + k] = c->group_ms[k];
  }
  return MMC_OK;
}

mmc_status mmc_fft_tuning(const mmc_ctx *c, int *variant, double ms[4]) {
  if (!c || !variant || !ms) return fail(MMC_ERR_ARG, "null argument");
  *variant = c->batch_plan.ready && c->batch_plan.il2d ? c->batch_plan.fft_variant : 0;
  for (int k = 0; k < 4; ++k) ms[k] = c->tune_ms[k];
  return MMC_OK;
}
int mmc_nchains(const mmc_ctx *c) { return c ? c->nchains : 0; }

mmc_status mmc_demag_kernel(const double h[3], const int n[3], const int periodic[3], int images, int ox, int oy,
                            int oz, double *out) {
  if (!h || !n || !periodic || !out) return fail(MMC_ERR_ARG, "null argument");
  for (int a = 0; a < 3; ++a) {
    if (!(h[a] > 0.0)) return fail(MMC_ERR_ARG, "cell size must be > 0");
    if (n[a] < 1) return fail(MMC_ERR_ARG, "extents must be >= 1");
  }
  if (images < 0 || images > kMaxDemagImages) return fail(MMC_ERR_ARG, "images must be in [0, 64]");
  if (ox < 1 || oy < 1 || oz < 1) return fail(MMC_ERR_ARG, "offset counts must be >= 1");
  if (1LL * ox * oy * oz > (1LL << 24)) return fail(MMC_ERR_ARG, "more than 2^24 offsets");
  DemagPeriodic pd;
  for (int a = 0; a < 3; ++a) {
    pd.n[a] = n[a];
    pd.per[a] = periodic[a] ? 1 : 0;
  }
  pd.images = images;
  std::vector<double> oct;
  demag_octant(h, ox, oy, oz, oct, pd);
  std::memcpy(out, oct.data(), oct.size() * sizeof(double));
  return MMC_OK;
}

mmc_status mmc_thermo(const double *T, int n, double Tc, double mu, double V, double Ms0, double sigma_cap,
                      double *me, double *chi, double *sigma, double *c2, double *c4) {
  if (n < 0 || (n > 0 && !T)) return fail(MMC_ERR_ARG, "need n >= 0 temperatures");
  if (!(Tc > 0.0) || !(V > 0.0) || !(Ms0 > 0.0)) return fail(MMC_ERR_ARG, "Tc, V and Ms0 must be > 0");
  if (!(sigma_cap > 0.0 && sigma_cap < 1.0)) return fail(MMC_ERR_ARG, "sigma_cap must be in (0, 1)");
  for (int i = 0; i < n; ++i)
    if (!(T[i] > 0.0)) return fail(MMC_ERR_ARG, "T must be > 0");
  const double m = mu > 0.0 ? mu : muB;
  for (int i = 0; i < n; ++i) {
    if (me) me[i] = me_of_T(T[i], Tc);
    if (chi) chi[i] = chi_of_T(T[i], Tc, m);
    if (sigma) sigma[i] = sigma_of_T(T[i], Tc, m, V, Ms0, sigma_cap);
    double a = 0.0, b = 0.0;
    long_coeffs(T[i], Tc, m, V, Ms0, &a, &b);
    if (c2) c2[i] = a;
    if (c4) c4[i] = b;
  }
  return MMC_OK;
}
int64_t mmc_ncell(const mmc_ctx *c, int chain) {
  if (!c || chain < 0 || chain >= c->nchains) return 0;
  return c->hc[chain].ncell;
}

struct CkptHeader {
  char magic[8];
  int32_t version, nchains;
  int64_t m_total;
  uint64_t host_sweep;
};

mmc_status mmc_checkpoint(mmc_ctx *c, void *buf, size_t *len) {
  if (!c || !len) return fail(MMC_ERR_ARG, "null argument");
  const size_t need = sizeof(CkptHeader) + (size_t)c->nchains * (sizeof(ChainState) + 3 * sizeof(float)) +
                      (size_t)c->m_total * sizeof(float4);
  if (!buf) {
    *len = need;
    return MMC_OK;
  }
  if (*len < need) return fail(MMC_ERR_ARG, "checkpoint buffer too small");
  char *p = (char *)buf;
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "MMCCKPT", 8);
  h.version = 1;
  h.nchains = c->nchains;
  h.m_total = c->m_total;
  h.host_sweep = c->host_sweep;
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  CUDA_TRY(cudaMemcpyAsync(p, c->d_st, (size_t)c->nchains * sizeof(ChainState), cudaMemcpyDeviceToHost, c->stream));
  p += (size_t)c->nchains * sizeof(ChainState);
  for (int i = 0; i < c->nchains; ++i) {
    const float B[3] = {c->ch[i].Bx, c->ch[i].By, c->ch[i].Bz};
    std::memcpy(p, B, sizeof(B));
    p += sizeof(B);
  }
  CUDA_TRY(cudaMemcpyAsync(p, c->d_m, (size_t)c->m_total * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  *len = need;
  return MMC_OK;
}

mmc_status mmc_restore(mmc_ctx *c, const void *buf, size_t len) {
  if (!c || !buf) return fail(MMC_ERR_ARG, "null argument");
  const size_t need = sizeof(CkptHeader) + (size_t)c->nchains * (sizeof(ChainState) + 3 * sizeof(float)) +
                      (size_t)c->m_total * sizeof(float4);
  if (len < need) return fail(MMC_ERR_ARG, "checkpoint too short");
  const char *p = (const char *)buf;
  CkptHeader h;
  std::memcpy(&h, p, sizeof(h));
  if (std::memcmp(h.magic, "MMCCKPT", 8) != 0 || h.version != 1 || h.nchains != c->nchains ||
      h.m_total != c->m_total)
    return fail(MMC_ERR_ARG, "checkpoint does not match this context");
  p += sizeof(h);
  CUDA_TRY(cudaMemcpyAsync(c->d_st, p, (size_t)c->nchains * sizeof(ChainState), cudaMemcpyHostToDevice, c->stream));
  p += (size_t)c->nchains * sizeof(ChainState);
  for (int i = 0; i < c->nchains; ++i) {
    float B[3];
    std::memcpy(B, p, sizeof(B));
    p += sizeof(B);
    c->ch[i].Bx = B[0]; c->ch[i].By = B[1]; c->ch[i].Bz = B[2];
    for (int a = 0; a < 3; ++a) c->hc[i].ecoef.B[a] = B[a];
  }
  CUDA_TRY(cudaMemcpyAsync(c->d_ch, c->ch.data(), c->ch.size() * sizeof(ChainDev), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->d_m, p, (size_t)c->m_total * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
  c->host_sweep = h.host_sweep;
  const unsigned base = (unsigned)h.host_sweep;
  CUDA_TRY(cudaMemcpyAsync(c->d_sweep_base, &base, sizeof(base), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->heff_stale = true;
  c->obs_fresh = false;
  return MMC_OK;
}

int mmc_checked_build(void) { return kChecked ? 1 : 0; }

mmc_status mmc_check_report(mmc_ctx *c, int64_t *count, int *site, int64_t range[3], int clear) {
  if (!c) return fail(MMC_ERR_ARG, "null context");
  MmcCheck r;
  std::memset(&r, 0, sizeof(r));
  if (c->d_check) {
    CUDA_TRY(cudaMemcpyAsync(&r, c->d_check, sizeof(r), cudaMemcpyDeviceToHost, c->stream));
    if (clear) CUDA_TRY(cudaMemsetAsync(c->d_check, 0, sizeof(MmcCheck), c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  if (count) *count = (int64_t)r.count;
  if (site) *site = r.count ? r.site : 0;
  if (range) {
    range[0] = r.index;
    range[1] = r.lo;
    range[2] = r.hi;
  }
  return MMC_OK;
}

mmc_status mmc_check_total(int64_t *count, int *site) {
  if (count) *count = (int64_t)g_check_total.load();
  if (site) *site = g_check_site.load();
  return MMC_OK;
}

const char *mmc_check_site_name(int site) {
  static const char *const names[kCkSiteCount] = {
      "none", "sweep block table", "sweep cell", "sweep neighbour", "sweep field", "sweep per-cell table",
      "sweep debug output", "band item", "band copy", "demag m", "demag spectrum", "demag tensor", "demag field",
      "demag block table", "fused copy", "fused state"};
  return site >= 0 && site < kCkSiteCount ? names[site] : "?";
}

const char *mmc_status_str(mmc_status s) {
  switch (s) {
    case MMC_OK: return "ok";
    case MMC_ERR_ARG: return "invalid argument";
    case MMC_ERR_CUDA: return "CUDA error";
    case MMC_ERR_TIMEOUT: return "device wait timed out";
    case MMC_ERR_NONFINITE: return "non-finite value";
    case MMC_ERR_UNSUPPORTED: return "unsupported combination";
    case MMC_ERR_NOMEM: return "out of memory";
  }
  return "unknown status";
}

const char *mmc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
