/*
 * mmc.h -- C ABI of a GB300 (sm_103a) implementation of the parallel
 * micromagnetic Monte Carlo (MMC) method of S. Lepadatu, "Micromagnetic Monte
 * Carlo method with variable magnetization length based on the
 * Landau-Lifshitz-Bloch equation" (arXiv:2106.05593).
 *
 * The problem statement follows the paper: a mesh of cells of volume V with
 * magnetization m = M/Ms0 (Sec. II), material parameters Ms0, A0 (exchange,
 * Eq. 10), D0 (interfacial DMI, Eq. 15), K1/K2 with easy axis e_A (uniaxial
 * Eq. 11, or cubic Eq. 12), Curie temperature Tc and atomic moment mu (Eqs. 8-9),
 * a temperature field T, an applied field, and the demagnetizing interaction by
 * FFT convolution with the Newell tensor (Sec. III, Eq. 14), open (zero padded)
 * or periodic in the plane (mmc_mesh.demag_images).
 * mmc_sweep runs MMC iterations: each cell, one checkerboard sublattice at a
 * time, proposes a rotation in a cone plus a multiplicative length change
 * (Sec. II) and accepts it with Eq. 5.
 *
 * Conventions shared by every entry point:
 *  - Every function returns mmc_status (MMC_OK == 0, errors < 0).  Nothing
 *    aborts, traps or throws across the ABI; mmc_status_str() gives text and
 *    mmc_last_error() the message of the last failure on the calling thread.
 *  - Units are SI: lengths in m, Ms0 in A/m, A0 in J/m, D0 in J/m^2, K in J/m^3,
 *    T and Tc in K, mu in J/T, applied fields as mu0*H in tesla.
 *  - Cell index q = i + nx*(j + ny*k) ("natural order").  Vector arrays of m
 *    exchanged with the caller are float4 per cell (x, y, z, unused) in natural
 *    order.
 *  - The library owns all device memory it allocates (cudaMalloc at create, freed
 *    at destroy).  Every pointer argument is a HOST pointer unless its comment
 *    says "device"; host buffers are owned by the caller and read or written
 *    only during the call.
 *  - Work is issued on the CUDA stream given at create (NULL = legacy default
 *    stream).  Calls that return results to host memory synchronize that stream.
 *  - A context holds nchains independent Markov chains ("batch"); a plain
 *    single-chain context is a batch of one.  Chains advance in lockstep: one
 *    sweep counter, one seed; Philox counter word 2 carries the chain index
 *    (plus mmc_options.chain_base).
 */
#ifndef MMC_H
#define MMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MMC_OK = 0,
    MMC_ERR_ARG = -1,         /* invalid argument (null, T <= 0, odd periodic extent, ...) */
    MMC_ERR_CUDA = -2,        /* a CUDA runtime / cuFFT call failed */
    MMC_ERR_TIMEOUT = -3,     /* a bounded device-side wait gave up (reported by mmc_observables) */
    MMC_ERR_NONFINITE = -4,   /* non-finite values in input or state */
    MMC_ERR_UNSUPPORTED = -5, /* a combination the library does not implement */
    MMC_ERR_NOMEM = -6        /* device or host allocation failed */
} mmc_status;

typedef struct mmc_ctx mmc_ctx;   /* opaque; owned by the library */

/* Mesh (Sec. II): nx*ny*nz cells; periodic[a] != 0 makes axis a periodic for the
 * exchange and DMI bonds and requires an even extent >= 2 on that axis.
 * demag_images selects the boundaries of the demagnetizing convolution (Eq. 14):
 * 0 open (zero padded) on every axis; P in [1, 64] periodic along every periodic
 * axis (the in-plane periodic films of Sec. III-IV), the kernel being the Newell
 * tensor summed over P periodic images on each side, each offset taken at its
 * minimal image and the half-period offset split evenly between its two minimal
 * images.  The periodic kernel is built on the host at create, at a cost that
 * grows as (2P + 1)^(periodic axes) tensor evaluations per offset; the device
 * work per update is the same as with open boundaries. */
typedef struct {
    int nx, ny, nz;
    int periodic[3];
    int demag_images;
} mmc_mesh;

/* Material (Sec. II-IV).  Scalars apply to every cell unless the matching
 * per-cell HOST array (ncell entries, natural order; e_A_cell: 3 per cell) is
 * non-NULL.  Temperature scaling: A and D enter as A0, D0 (the paper's
 * A/Me^2 = A0/Ms0^2); K1(T) = K1 m_e^3 and K2(T) = K2 m_e^10 for uniaxial,
 * K1 m_e^10 and K2 m_e^21 for cubic anisotropy (m_e^{l(l+1)/2}). */
typedef struct {
    double Ms0;               /* A/m */
    double A0;                /* J/m */
    double D0;                /* J/m^2, interfacial DMI (in-plane bonds) */
    double K1, K2;            /* J/m^3 at T = 0 */
    double e_A[3];            /* uniaxial easy axis (normalized by the library) */
    double Tc;                /* K */
    double mu_atom;           /* J/T in Eq. 8; <= 0 selects one Bohr magneton */
    int aniso_cubic;          /* 0 uniaxial (Eq. 11), 1 cubic along x, y, z (Eq. 12) */
    const double *Ms0_cell;   /* optional per-cell Ms0 */
    const double *K1_cell;    /* optional per-cell K1 */
    const double *e_A_cell;   /* optional per-cell easy axis, 3 per cell */
    const double *Tc_cell;    /* optional per-cell Tc */
    const int *grain;         /* optional grain id per cell */
    double grain_exch_scale;  /* exchange and DMI scale of bonds joining two grains */
} mmc_material;

/* Options.  mmc_default_options() fills the documented defaults. */
typedef struct {
    int demag;                /* 1: include the demag interaction (Eq. 14)          [0] */
    int demag_per_pass;       /* 1: recompute H_d before each sublattice pass       [0] */
    int demag_fp64;           /* precision of the sweep's FFT convolution:          [0]
                                 0 FP32; 1 FP64; 2 float-float (pairs of FP32 values,
                                 ~48-bit significands, on the FP32 pipe).  Energies
                                 and mmc_demag_field always use FP64. */
    int demag_cufft;          /* 1: cuFFT R2C/C2R transforms (comparison path) for the
                                 sweep's demag field instead of the own kernels [0] */
    int adapt;                /* 1: adapt the cone angle every 100 sweeps (Sec. II) [1] */
    double theta0_deg;        /* initial cone half-angle                           [30] */
    double sigma_cap;         /* cap of Eq. 13                                   [0.03] */
    int hist_bins;            /* |m| histogram bins on [0, hist_max)              [200] */
    double hist_max;          /*                                                    [1] */
    int use_graphs;           /* 1: capture 100-sweep blocks in CUDA graphs         [1] */
    int stream_groups;        /* chain groups whose iterations run concurrently on
                                 their own streams, so that one group's kernel tails
                                 overlap the other's work; 0 auto (1, 2 or 3 groups,
                                 timed on the batch at create, see mmc_tuning), 1
                                 one stream, G > 1 G groups.  Results are
                                 identical for any value.                        [0] */
    int demag_self;           /* serial form (mmc_sweep_serial) only: add the demag
                                 self term (mu0 V / 2) Ms0^2 dm.N(0).dm to Eq. 14,
                                 making its demag energy change exact           [0] */
    int fft_variant;          /* FP32 2D demag kernels: 0 time the variants on the
                                 batch at create and keep the fastest, 1 radix 16
                                 (768 threads), 2 radix 32 (384 threads), 3 radix
                                 16 (384 threads, two blocks per SM), 4 one warp
                                 per 1024-point sequence as a 32 x 32 split (only
                                 when every chain's padded grid is 1024 x 1024 and
                                 open; otherwise 1)                              [0] */
    int demag_stripes;        /* S > 1: each sublattice pass runs in S bands of rows
                                 (j + ny k in [floor(b nrows / S), floor((b+1)
                                 nrows / S))), the demag field recomputed before
                                 every band: a schedule between demag before each
                                 pass and the serial form (App. B).  0 or 1: whole
                                 passes (demag_per_pass decides).                [1] */
    int chain_base;           /* Philox counter word 2 of chain c is chain_base + c
                                 (>= 0, chain_base + nchains < 2^31): a one-chain
                                 context with chain_base = c draws the random
                                 numbers of chain c of a batch, so the plain and
                                 batched forms of the same chain are the same
                                 Markov chain, bit for bit.                      [0] */
    int sweep_tiles;          /* 1: batches whose chains are all one cell thick,
                                 with uniform material and at most 1024 cells per
                                 row, run the sublattice pass on shared-memory
                                 halo tiles: bands of rows brought in by bulk
                                 asynchronous copies while the previous band is
                                 computed; 0: the per-block pass.  The same
                                 moves either way, up to the last-bit rounding of
                                 the energy terms (separately compiled kernels;
                                 each is deterministic on its own).  On GB300
                                 the per-block pass is faster for these chains
                                 (the pass is bound by instruction issue, and
                                 the banded kernel holds more registers).       [0] */
    int wait_polls;           /* bound of a kernel's wait for its copies, in polls
                                 of the barrier (0: 2^22, about a second); a wait
                                 that runs out skips its band and makes the next
                                 mmc_observables return MMC_ERR_TIMEOUT          [0] */
    int wait_test;            /* test hook for that path: 1 makes every band wait
                                 for 16 bytes that no copy delivers, so every wait
                                 runs out (no band is updated)                  [0] */
    int fuse_passes;          /* 1: batches of uniform one-cell-thick chains on the
                                 1024 x 1024 warp-transform demag kernels (FFT
                                 variant 4) run the inverse row transforms with
                                 the red pass, and the black pass with the next
                                 iteration's forward row transforms, as one kernel
                                 per tile of four rows each (a tile's red cells
                                 can move once its field is known, its rows are
                                 final once their black cells moved); 0: separate
                                 kernels.
                                 The same moves either way, up to the last-bit
                                 rounding of separately compiled kernels.       [1] */
} mmc_options;

/* One chain of a batch. T_cell (optional, HOST) gives a per-cell temperature;
 * otherwise T applies to all cells.  B is the applied field (tesla). */
typedef struct {
    mmc_mesh mesh;
    double cellsize[3];
    mmc_material material;
    double T;
    const double *T_cell;
    double B[3];
} mmc_chain_desc;

/* Observables (Sec. II, Figs. 1-2): averages over the snapshots accumulated by
 * mmc_sweep_sampled since the last reset, or over the current state when none.
 * hist (optional HOST buffer of hist_bins + 1 counters, last = overflow) is
 * filled with the |m| histogram of the same samples. */
typedef struct {
    double mean_m[3];         /* <m> */
    double mean_len;          /* <|m|> */
    double mean_len2;         /* <|m|^2> */
    int64_t nsnap;            /* snapshots averaged (0: current state) */
    int64_t nonfinite;        /* cells with a non-finite component */
    double acc_rate;          /* acceptance rate of the last completed 100-sweep window */
    double theta_deg;         /* current cone half-angle */
    int64_t sweeps;           /* sweep counter */
    int64_t *hist;            /* optional, hist_bins + 1 entries */
} mmc_obs;

/* ---------------------------------------------------------------------------
 * Lifetime
 * ------------------------------------------------------------------------- */

/* Fill *opt with the defaults shown in brackets above. */
mmc_status mmc_default_options(mmc_options *opt);

/* Create a context of nchains chains (Sec. II-IV problem statement).
 * Validates the inputs (MMC_ERR_ARG: null pointers, non-positive sizes or
 * temperatures, odd periodic extents, FFT sizes above 4096), computes the
 * thermodynamic tables m_e(T), chi(T) (Eqs. 8-9) and sigma (Eq. 13), the Newell
 * tensor spectra (Eq. 14, FP64 on the host) and uploads everything once.  The
 * initial state is m = m_e(T) along +x per cell (or 0.3 where m_e = 0); use
 * mmc_set_m / mmc_init_random to change it.  cuda_stream is a cudaStream_t or
 * NULL.  On success *out owns device memory until mmc_destroy. */
mmc_status mmc_create(const mmc_chain_desc *chains, int nchains, const mmc_options *opt,
                      void *cuda_stream, mmc_ctx **out);

/* Convenience for one chain: mesh, cell size, material, T (scalar, or T_cell).
 * Same semantics as mmc_create with nchains = 1 and zero applied field. */
mmc_status mmc_create_single(const mmc_mesh *mesh, const double cellsize[3],
                             const mmc_material *mat, double T, const double *T_cell,
                             const mmc_options *opt, void *cuda_stream, mmc_ctx **out);

/* Release every resource of ctx (NULL is accepted). */
void mmc_destroy(mmc_ctx *ctx);

/* ---------------------------------------------------------------------------
 * State
 * ------------------------------------------------------------------------- */

/* Applied field of one chain (chain < 0: all chains), tesla. */
mmc_status mmc_set_field(mmc_ctx *ctx, int chain, const double B[3]);

/* Temperature of one chain (chain < 0: all chains), kelvin: recomputes the
 * temperature-dependent tables exactly as at create -- m_e(T), chi(T) (Eqs. 8-9),
 * sigma (Eq. 13), the longitudinal coefficients of Eq. 7, K(T) ~ m_e^{l(l+1)/2}
 * and the kT-unit coefficients of the sweep -- and leaves the state, the sweep
 * counter and the cone angle alone.  T_cell (optional HOST, ncell values in
 * natural order, one chain only) gives per-cell temperatures to a chain that
 * has per-cell tables (MMC_ERR_UNSUPPORTED otherwise).  MMC_ERR_ARG: T <= 0 or
 * a non-positive T_cell value. */
mmc_status mmc_set_temperature(mmc_ctx *ctx, int chain, double T, const double *T_cell);

/* Copy m of one chain in/out as float4 per cell in natural order.  src/dst are
 * HOST pointers when is_device == 0, DEVICE pointers otherwise; the caller's
 * buffer is no longer used when the call returns.  mmc_set_m rejects non-finite
 * values (MMC_ERR_NONFINITE, state unchanged; checked on the device).  The demag
 * field is not recomputed here: every iteration of mmc_sweep / mmc_sweep_serial
 * computes it first, and mmc_pass_debug refreshes it when the state or the
 * field changed since the last update (mmc_demag_update forces it). */
mmc_status mmc_set_m(mmc_ctx *ctx, int chain, const float *src, int is_device);
mmc_status mmc_get_m(mmc_ctx *ctx, int chain, float *dst, int is_device);

/* The same for every chain of the batch in one call (the batched form of
 * Sec. II's parallel algorithm: one copy and one check instead of one per
 * chain): src/dst hold chain 0's cells in natural order, then chain 1's, and so
 * on (sum of the chains' cells x 4 floats).  mmc_set_m_all rejects the whole
 * batch if any value is non-finite (MMC_ERR_NONFINITE, no chain changed).  The
 * first call allocates a device buffer of that size (MMC_ERR_NOMEM if it
 * cannot); the caller's buffer is no longer used when the call returns. */
mmc_status mmc_set_m_all(mmc_ctx *ctx, const float *src, int is_device);
mmc_status mmc_get_m_all(mmc_ctx *ctx, float *dst, int is_device);

/* Random initial directions from Philox counter (cell, 0, chain, 1), key seed:
 * z = 2 u0 - 1, phi = 2 pi u1, length len (len <= 0: m_e, or the Eq. 7 rms
 * length where m_e = 0). */
mmc_status mmc_init_random(mmc_ctx *ctx, uint64_t seed, double len);

/* ---------------------------------------------------------------------------
 * Monte Carlo (Sec. II, III)
 * ------------------------------------------------------------------------- */

/* n MMC iterations of every chain.  Each iteration: (demag field, Eq. 14, if
 * enabled) -> red pass ((i+j+k) even) -> [demag again if demag_per_pass] ->
 * black pass; every 100 iterations of the global counter the cone angle is
 * adapted (Sec. II).  Random numbers: Philox4x32-10 with counter
 * (cell, sweep, chain, 0) and key (seed & 0xffffffff, seed >> 32); uniforms
 * ((r >> 9) + 1/2) 2^-23.  Runs entirely on the device. */
mmc_status mmc_sweep(mmc_ctx *ctx, int64_t n, uint64_t seed);

/* As mmc_sweep, accumulating an observable snapshot every sample_every
 * iterations (sample_every >= 1) into device accumulators read by
 * mmc_observables. */
mmc_status mmc_sweep_sampled(mmc_ctx *ctx, int64_t n, uint64_t seed, int sample_every);

/* Recompute the demag field of every chain from the current state (Eq. 14). */
mmc_status mmc_demag_update(mmc_ctx *ctx);

/* n MMC iterations of the serial form of the method (App. B) on every chain:
 * the cells are visited one at a time in index order i + nx (j + ny k); a move's
 * demag energy change is exact, the frozen-field term of Eq. 14 plus the self
 * term (mu0 V / 2) Ms0^2 dm . N(0) . dm, and after every accepted move the demag
 * field of the whole chain is updated by -N(r - q) . dM_q (Newell tensor N), so
 * every move sees the field of the current state.  The field is recomputed by
 * the FFT convolution at the start of every iteration (in the precision of
 * mmc_options.demag_fp64; later updates in FP32).  Philox counters, moves,
 * acceptance rule (Eq. 5), sweep counter and cone adaptation are those of
 * mmc_sweep, so the same seed gives the same random numbers per cell and
 * iteration in both forms.  Without demag this is the serial index-order
 * Metropolis sweep.  One thread block per chain, O(N^2) work per iteration:
 * meant for small chains (the comparison of App. B).  Chains whose moments,
 * field and tensor fit in 200 KB (48 B per cell in 2D, 56 B in 3D, about
 * 4,200 cells in 2D) run from shared memory, larger ones from global memory.
 * demag_per_pass has no meaning here; options.use_graphs is not used. */
mmc_status mmc_sweep_serial(mmc_ctx *ctx, int64_t n, uint64_t seed);

/* One sublattice pass of one chain with explicit sweep index and cone angle,
 * leaving the sweep counter, the adaptation window and the other chains alone:
 * diagnostic form used by parity checks.  Accepted moves are written to the
 * chain's state, as in mmc_sweep.  dec (optional HOST, ncell floats) receives the decision value
 * d = dF/kT - 4 ln(m'/m) + ln u3 (accept iff d < 0) of the cells of that
 * colour, acc (optional HOST, ncell int8) 1/0 for them and -1 for the others. */
mmc_status mmc_pass_debug(mmc_ctx *ctx, int chain, int color, uint32_t sweep, uint64_t seed,
                          double theta_deg, float *dec, int8_t *acc);

/* ---------------------------------------------------------------------------
 * Measurements
 * ------------------------------------------------------------------------- */

/* Observables of one chain (see mmc_obs); reset != 0 clears the snapshot
 * accumulators after reading them. */
mmc_status mmc_observables(mmc_ctx *ctx, int chain, mmc_obs *out, int reset);

/* Observables of every chain in one device round trip: out[k] (k < nchains,
 * HOST array) receives what mmc_observables(ctx, k, &out[k], reset) would, each
 * out[k].hist optional as there; reset != 0 clears the snapshot accumulators
 * of every chain.  MMC_ERR_TIMEOUT as for mmc_observables (out not filled). */
mmc_status mmc_observables_all(mmc_ctx *ctx, mmc_obs *out, int reset);

/* Angular-deviation histogram of one chain's current state (Sec. II, Fig. 1d-f):
 * the polar angle of every cell to the chain's mean direction, counted in `bins`
 * equal bins on [theta_lo, theta_hi) (radians, 1 <= bins <= 1024); angles outside
 * go to hist[bins].  The paper bins each configuration between its own minimum
 * and maximum angle and averages over ensembles; averaging needs common bins, so
 * the range is the caller's.  hist: HOST, bins + 1 counters; mean_dir (optional
 * HOST) receives the unit mean direction.  Angles in FP64 of the FP32 state. */
mmc_status mmc_angle_hist(mmc_ctx *ctx, int chain, int bins, double theta_lo, double theta_hi, int64_t *hist,
                          double mean_dir[3]);

/* Size of the free-energy terms of the trial moves (App. B, Fig. 11): for every
 * cell of one chain, both sublattices evaluated against the current state and
 * its frozen demag field (Eq. 14), the trial move the sweep would draw at
 * iteration `sweep` with `seed` (Philox counter (cell, sweep, chain, 0), cone
 * half-angle theta_deg, or the chain's current angle when theta_deg < 0, and the
 * length move of Eq. 13) is formed and its free-energy change split by term.
 * out[6] (HOST) receives the means over the cells of |dF| / kT of the cell:
 * exchange (Eq. 10), DMI (Eq. 15), anisotropy (Eqs. 11-12), Zeeman, longitudinal
 * (Eq. 7), demag (Eq. 14).  The state is not changed; averaging the result over
 * the states of a run gives the paper's per-term averages.  MMC_ERR_ARG:
 * theta_deg > 180 or a null output. */
mmc_status mmc_trial_terms(mmc_ctx *ctx, int chain, uint32_t sweep, uint64_t seed, double theta_deg,
                           double out[6]);

/* Energy terms of one chain, in J: out[7] = {total, exchange, dmi, anisotropy,
 * zeeman, longitudinal (Eq. 7), demag (E_d = -(mu0 V/2) sum Ms0 m.H_d)}.
 * Sums accumulate in FP64; the demag field of the current state is recomputed
 * with the FP64 convolution. */
mmc_status mmc_energy(mmc_ctx *ctx, int chain, double out[7]);

/* Demag field H_d (A/m) of one chain's current state, 3 doubles per cell in
 * natural order (HOST), from the FP64 convolution. */
mmc_status mmc_demag_field(mmc_ctx *ctx, int chain, double *H);

/* The demag field H_d (A/m) the sweep itself uses for one chain (Sec. III,
 * Eq. 14): the context's own convolution of the current state, with the FFT
 * kernels and precision the sweep runs (FP32 unless demag_fp64, the FFT variant
 * of mmc_fft_tuning), 3 doubles per cell in natural order (HOST).  A diagnostic
 * of the precision of the sweep's frozen field; MMC_ERR_UNSUPPORTED on the cuFFT
 * comparison path (demag_cufft). */
mmc_status mmc_sweep_field(mmc_ctx *ctx, int chain, double *H);

/* Thermodynamic tables of one chain (HOST, ncell doubles each, any may be NULL):
 * m_e (Eq. 9), chi (Eq. 8, 1/T), sigma (Eq. 13 capped). */
mmc_status mmc_tables(mmc_ctx *ctx, int chain, double *me, double *chi, double *sigma);

/* Differentiable form: energy and hand-written gradient of one chain for a
 * caller-given state (Eqs. 7, 10, 11, 12, 14, 15).  m is a DEVICE array of
 * 3*ncell values in natural order, double if fp64 != 0 else float.  params
 * (HOST, optional) = {Ms0, A0, D0, Ku, chi} overrides the chain's material for
 * this call: Ms0 (A/m), A0 (J/m), D0 (J/m^2), the T = 0 anisotropy constant Ku
 * (K1(T) = Ku m_e^3) and the longitudinal susceptibility chi (1/T) of Eq. 7;
 * NULL uses the chain's own values.  E (HOST, 7 doubles) receives the terms as
 * mmc_energy; dEdm (DEVICE, optional, same type and size as m) dE/dm_i in J per
 * unit m; dEdp (HOST, optional, 5 doubles) dE/d{Ms0, A0, D0, Ku, chi}.  The
 * demag field is recomputed from m by the FFT convolution in the requested
 * precision on every call; nothing is kept between calls.  Chains with per-cell
 * material or temperature return MMC_ERR_UNSUPPORTED. */
mmc_status mmc_energy_grad(mmc_ctx *ctx, int chain, const void *m, int fp64, const double params[5],
                           double E[7], void *dEdm, double dEdp[5]);

/* Zero-temperature steepest descent on one chain, the comparison method of
 * Sec. III (SDesc): the energy of mmc_energy (exchange, DMI, anisotropy,
 * Zeeman, demag; the longitudinal term vanishes at |m| = m_e) is minimized over
 * the directions u_i with every |m_i| held at m_e(T), i.e. with the parameters
 * rescaled to T and no stochasticity or length distribution.  Steps
 * u_i <- normalize(u_i - tau g_i), g_i the tangential gradient m_e (G_i - (G_i.u_i) u_i)
 * of G = dE/dm (FP64, as mmc_energy_grad); tau turns the steepest cell by 0.01 rad
 * on the first step, then alternates the Barzilai-Borwein sizes s.s/s.y and
 * s.y/y.y (s, y the changes of u and g; the previous tau is kept when s.y <= 0).
 * Stops when the largest normalized torque |u_i x h_i| / |h_i|, h = -m_e G, is
 * below tol (the paper uses 1e-5) or after maxit steps; the chain's state is
 * replaced by the result.  Outputs (HOST, each may be NULL): steps taken, final
 * largest torque (compare with tol to see convergence), energy terms E[7] of the
 * result as mmc_energy.  Uniform chains below Tc only (MMC_ERR_UNSUPPORTED for
 * per-cell material, MMC_ERR_ARG at or above Tc). */
mmc_status mmc_minimize(mmc_ctx *ctx, int chain, int64_t maxit, double tol, int64_t *iters, double *torque,
                        double E[7]);

/* Per-kernel timing: runs n MMC iterations eagerly (as mmc_sweep, without
 * graphs) with CUDA events recorded on the context's stream around every kernel
 * and returns, per kernel kind, the summed duration in ms (ms) and the number
 * of launches (count).  Kinds: 0 demag rows forward, 1 demag columns, 2 demag
 * rows inverse, 3 sublattice pass, 4 observables, 5 window/adaptation step,
 * 6 black pass fused with the forward rows, 7 inverse rows fused with the red
 * pass (mmc_options.fuse_passes; kind 0 is then the forward rows that start each
 * block of iterations).  Both arrays have 8 entries (HOST). */
mmc_status mmc_phase_times(mmc_ctx *ctx, int64_t n, uint64_t seed, double ms[8], int64_t count[8]);

/* FFT variant of the batch's FP32 2D demag kernels (1 radix 16 with 768-thread
 * blocks, 2 radix 32 with 384-thread blocks, 3 radix 16 with 384-thread blocks,
 * two per SM, 4 warp-resident 32 x 32 transforms for batches whose padded grids
 * are all 1024 x 1024; 0 when the batch does not use them) and, when
 * mmc_options.fft_variant was 0, the per-update times in ms that the
 * create-time timing measured for the four variants (ms has 4 entries; 0 for a
 * variant that was not timed).  The variants compute the same convolution with FP32 rounding in
 * a different order, so the demag field, and through it the chain, can differ
 * between them at rounding level; set the variant explicitly where runs must
 * repeat bit for bit across contexts.  (HOST outputs.)  Not a paper quantity: a
 * tuning record of this implementation. */
mmc_status mmc_fft_tuning(const mmc_ctx *ctx, int *variant, double ms[4]);

/* The create-time autotuner's picks: the FFT variant (as mmc_fft_tuning), the
 * number of chain groups on concurrent streams, and whether both came from the
 * tuning cache (1) or were timed on the batch (0).  ms (optional, 7 doubles):
 * per-update times of FFT variants 1..4 and per-iteration times with 1, 2, 3
 * groups, as timed (0 where not timed).  The cache is a text file, one line per
 * problem, named by the environment variable MMC_TUNE_CACHE ("" or "off"
 * disables it), by default $XDG_CACHE_HOME/mmc_gb300/tune.txt or
 * ~/.cache/mmc_gb300/tune.txt; its key is the GPU model and a hash of the
 * chains' extents, periodicity, demag images and per-cell flag and of the
 * kernel-selecting options.  A second create of the same problem reads the
 * picks instead of timing, so both contexts run the same kernels.  (HOST
 * outputs; a tuning record of this implementation, not a paper quantity.) */
mmc_status mmc_tuning(const mmc_ctx *ctx, int *fft_variant, int *stream_groups, int *from_cache, double ms[7]);


/* Number of kernels the library launched since create (all kinds). */
int64_t mmc_kernel_launches(const mmc_ctx *ctx);

/* Number of chains and cells of a chain. */
int mmc_nchains(const mmc_ctx *ctx);
int64_t mmc_ncell(const mmc_ctx *ctx, int chain);

/* The demag kernel the library convolves with (Sec. III, Eq. 14), computed on the
 * host in FP64 without a context or a GPU: the Newell tensor of cells of size h
 * (m) at cell offsets (x, y, z), 0 <= x < ox, 0 <= y < oy, 0 <= z < oz, or, along
 * the axes with periodic[a] != 0 and images > 0, its sum over `images` periodic
 * images of extent n[a] on each side (mmc_mesh.demag_images).  out (HOST,
 * 6 ox oy oz doubles) receives xx yy zz xy xz yz of offset (x, y, z) at
 * out[6 (x + ox (y + oy z)) + c].  MMC_ERR_ARG: null pointers, non-positive
 * sizes, extents or counts, images outside [0, 64], more than 2^24 offsets. */
mmc_status mmc_demag_kernel(const double h[3], const int n[3], const int periodic[3], int images, int ox, int oy,
                            int oz, double *out);

/* The thermodynamic tables the library builds (Sec. II), computed on the host in
 * FP64 without a context or a GPU: for each of n temperatures T[i] (K), m_e
 * (Eq. 9), chi (Eq. 8, 1/T), the length-move width sigma (Eq. 13, capped at
 * sigma_cap, the cap at and above Tc) and the coefficients c2, c4 of the Eq. 7
 * free energy F = c2 m^2 + c4 m^4 + const (J) of a cell of volume V (m^3) with
 * Ms0 (A/m), Curie temperature Tc and atomic moment mu (J/T; <= 0: one Bohr
 * magneton).  Output arrays (HOST, n values) may be NULL.  MMC_ERR_ARG: T <= 0,
 * Tc, V or Ms0 <= 0, sigma_cap outside (0, 1), n < 0, a null T with n > 0. */
mmc_status mmc_thermo(const double *T, int n, double Tc, double mu, double V, double Ms0, double sigma_cap,
                      double *me, double *chi, double *sigma, double *c2, double *c4);

/* Checkpoint: serialize the full chain state (m of all chains, sweep counter,
 * cone angle, window counters, applied fields) into buf.  With buf == NULL only
 * *len is set to the required size.  mmc_restore accepts a buffer from a context
 * created with the same chain descriptors; resuming reproduces the
 * uninterrupted run bit for bit. */
mmc_status mmc_checkpoint(mmc_ctx *ctx, void *buf, size_t *len);
mmc_status mmc_restore(mmc_ctx *ctx, const void *buf, size_t len);

/* Observables of a caller-owned state, with no device allocation by the
 * library.  The paper has no counterpart: this is a service entry point for
 * callers that cannot allocate device memory themselves or through a library
 * call -- code recording a CUDA graph (an allocation breaks the capture),
 * frameworks whose caching allocator owns all device memory, and latency-
 * critical loops that cannot pay the implicit synchronization of cudaMalloc.
 * It computes the same quantities as mmc_observables (current state):
 *   m    DEVICE, n float4 (mx, my, mz, unused) cells, any order;
 *   out  DEVICE, 8 doubles: <mx>, <my>, <mz>, <|m|>, <|m|^2> over the finite
 *        cells, the number of non-finite cells, the number of finite cells, 0;
 *   hist DEVICE, hist_bins + 1 counters of |m| on [0, hist_max) (last =
 *        overflow), cleared by the call.
 * m must be 16-byte aligned and out, hist 8-byte aligned (MMC_ERR_ARG
 * otherwise, with nothing launched).
 * Work is queued on cuda_stream (a cudaStream_t of the current device, or NULL
 * for the legacy stream; a stream of another device is MMC_ERR_ARG); the call
 * does not synchronize.  Scratch for the per-block partial
 * sums is a fixed 128 KiB __device__ array inside the library, so n is limited
 * to 2,097,152 cells (MMC_ERR_ARG beyond that, with nothing launched).  The
 * first call on each device looks up that array's device address with the
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use this entry point after a
 * reset of the device (cudaDeviceReset), which invalidates the kept address.  All calls
 * on a device share the array: calls whose kernels may overlap on the GPU
 * (different streams without ordering) race and give wrong results.  Every
 * call overwrites the partials it reads, so no clearing is needed between
 * calls. */
mmc_status mmc_observables_noalloc(const float *m, int64_t n, int hist_bins, double hist_max,
                                   double *out, unsigned long long *hist, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Bounds-checked builds (no counterpart in the paper: a debugging aid in place
 * of a memory checker).  A library built with -DMMC_CHECKED (build.py,
 * build(checked=True): libmmc_checked.so) compares every global-memory index
 * of the sweep and demag kernels with the range of the buffer region it
 * belongs to before the access; an index outside is counted, the first one is
 * recorded, and the access goes to the first element of the region instead,
 * so a wrong index is reported here and never faults.  Normal builds carry no
 * checks and always report zero.
 * ------------------------------------------------------------------------- */

/* 1 in a checked build, 0 otherwise.  Host only. */
int mmc_checked_build(void);

/* The out-of-range indices met since the context was created or last cleared:
 * *count of them; for the first, *site (see mmc_check_site_name), and
 * range[0] = the index, range[1..2] = the range [lo, hi) it had to lie in
 * (element units of the buffer, relative as the kernel indexes it).  Any output
 * pointer may be NULL.  clear != 0 resets the record after reading it.
 * Synchronizes the context's stream. */
mmc_status mmc_check_report(mmc_ctx *ctx, int64_t *count, int *site, int64_t range[3], int clear);

/* The out-of-range indices met by all contexts destroyed so far in this
 * process (checked builds; 0 otherwise), and the site of the first of them.
 * Host only. */
mmc_status mmc_check_total(int64_t *count, int *site);

/* Name of an access site of mmc_check_report ("?" for an unknown one). */
const char *mmc_check_site_name(int site);

const char *mmc_status_str(mmc_status s);
const char *mmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MMC_H */
