/*
 * mmc_oracle.h -- plain, slow, serial FP64 CPU oracle of the micromagnetic
 * Monte Carlo (MMC) method of Lepadatu, "Micromagnetic Monte Carlo method with
 * variable magnetization length based on the Landau-Lifshitz-Bloch equation"
 * (arXiv:2106.05593).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA product path.
 *
 * Every function follows a passage of the paper, cited by section / equation:
 *   Eq. 1-5   acceptance rule with the m^4 length factor (Sec. II)
 *   Eq. 7     longitudinal free energy, both sides of Tc (Sec. II)
 *   Eq. 8, 9  longitudinal susceptibility and equilibrium magnetization (Sec. II)
 *   Eq. 10    exchange (factor 2 restored per vector)        (Sec. II)
 *   Eq. 11    uniaxial anisotropy                            (Sec. II)
 *   Eq. 12    cubic anisotropy                               (Sec. II)
 *   Eq. 13    length-move width sigma, capped at 0.03        (Sec. II)
 *   Eq. 14    demagnetizing field by convolution with the demag tensor and the
 *             frozen-field energy change                     (Sec. III); periodic
 *             along pbc axes as a truncated sum over images  (Sec. III, films)
 *   Eq. 15    interfacial DMI                                (Sec. IV)
 *   Sec. II   MMC iteration: cone rotation + length change, red-black passes,
 *             cone angle adapted every 100 iterations by +-1 deg outside 0.5+-0.05
 *   App. B    serial MMC with the demag field updated after every accepted move;
 *             the per-term size of the trial moves' free-energy changes (Fig. 11)
 *
 * Parity status of each function (what pins it) is listed in the header
 * comment of mmc_oracle.c.
 */
#ifndef MMC_ORACLE_H
#define MMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* CODATA 2018 SI constants */
#define ORC_KB   1.380649e-23
#define ORC_MUB  9.2740100783e-24
#define ORC_MU0  1.25663706212e-6

/* Problem statement (Sec. II-IV): mesh, cell size, material, temperature, field.
 * All per-cell arrays have ncell = nx*ny*nz entries in natural order
 * i + nx*(j + ny*k); eA has 3*ncell entries. They are copied by orc_create. */
typedef struct {
    int nx, ny, nz;
    int pbc[3];                 /* periodic flags; a periodic extent must be even */
    double h[3];                /* cell size (m) */
    double A0;                  /* exchange stiffness at T=0 (J/m); A/Me^2 = A0/Ms0^2 */
    double D0;                  /* interfacial DMI at T=0 (J/m^2) */
    double mu;                  /* atomic moment in Eq. 8 (J/T) */
    double sigma_cap;           /* cap of Eq. 13 (0.03 in the paper) */
    double grain_exch_scale;    /* exchange / DMI scale of bonds between grains */
    double B[3];                /* applied field mu0*H (T) */
    int demag;                  /* include the demagnetizing interaction */
    int demag_self;             /* add the exact self term to the frozen-field dF_d */
    int len_power;              /* power of m_B/m_A in Eq. 5; the paper's value is 4 */
    int aniso_cubic;            /* 0: uniaxial (Eq. 11), 1: cubic (Eq. 12) */
    const double *Ms0;          /* zero-temperature saturation magnetization (A/m) */
    const double *K1;           /* first anisotropy constant at T=0 (J/m^3) */
    const double *K2;           /* second anisotropy constant at T=0 (J/m^3) */
    const double *eA;           /* uniaxial easy axis (unit), 3 per cell */
    const double *Tc;           /* Curie temperature (K) */
    const double *T;            /* temperature (K) */
    const int *grain;           /* grain id per cell, or NULL for a single grain */
    uint32_t cell_base;         /* natural index of this mesh's first cell in a larger
                                   lattice it is a window of (the Philox counter word 0
                                   is the cell's index in the whole lattice); 0 normally */
    int demag_images;           /* > 0: the demag convolution is periodic along every
                                   pbc axis, summed over this many periodic images on
                                   each side (the in-plane periodic films of
                                   Sec. III-IV); 0: open boundaries */
} orc_problem;

typedef struct orc_ctx orc_ctx;

/* Observable accumulator (Sec. II, Fig. 1-2: length distribution, mean m). */
typedef struct {
    double sum_m[3];
    double sum_len, sum_len2;
    int64_t nsamples;           /* cell samples */
    int64_t nsnap;              /* snapshots */
    int64_t *hist;              /* hist_bins + 1 (overflow) counters, caller-owned */
    int hist_bins;
    double hist_max;
} orc_obs;

/* ---- random numbers: Philox4x32-10 (Salmon et al., SC'11) -------------- */
void   orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t r);

/* ---- thermodynamic functions (Eqs. 7-9, 13) ---------------------------- */
double orc_langevin(double x);
double orc_langevin_d(double x);
double orc_me(double T, double Tc);
double orc_chi(double T, double Tc, double mu);
double orc_sigma(double T, double Tc, double mu, double V, double Ms0, double cap);
double orc_long_energy(double m, double T, double Tc, double mu, double V, double Ms0);

/* ---- demagnetizing tensor (Newell) -------------------------------------- */
void orc_newell(double dx, double dy, double dz, double X, double Y, double Z, double out[6]);
void orc_tensor_quad(double dx, double dy, double dz, double X, double Y, double Z,
                     int npts, double out[6]);
void orc_tensor(double dx, double dy, double dz, double X, double Y, double Z, double out[6]);
/* demag kernel at cell offset (X, Y, Z) of the problem: the tensor, or along
 * periodic demag axes the sum over images (see orc_problem.demag_images) */
void orc_kernel(const orc_ctx *c, int X, int Y, int Z, double out[6]);

/* ---- context ------------------------------------------------------------ */
orc_ctx *orc_create(const orc_problem *p);
void     orc_destroy(orc_ctx *c);
int      orc_ncell(const orc_ctx *c);
void     orc_set_field(orc_ctx *c, const double B[3]);
void     orc_tables(const orc_ctx *c, double *me, double *chi, double *sigma,
                    double *K1T, double *K2T);

/* demag field H_d (A/m) of state m (3*ncell), method 0: direct sum, 1: FFT */
void orc_demag_field(orc_ctx *c, const double *m, double *H, int method);
/* full energy terms (J): [total, exchange, dmi, anisotropy, zeeman, longitudinal, demag] */
void orc_energy(orc_ctx *c, const double *m, double out[7]);
/* per-vector free energies summed over cells: Eq. 10, Eq. 15, Eq. 14 (J) */
void orc_pervector_sums(orc_ctx *c, const double *m, double out[3]);
/* energy change of cell i for m_i -> mnew (J): [total, ex, dmi, an, zee, long, demag(frozen)] */
void orc_local_dF(orc_ctx *c, const double *m, const double *H, int i,
                  const double mnew[3], double out[7]);
/* analytic gradient dE/dm (J per unit m, 3*ncell) and
 * dE/d(Ms0, A0, D0, Ku, chi) for uniform material; E[7] as orc_energy */
void orc_energy_grad(orc_ctx *c, const double *m, double *dEdm, double dEdp[5], double E[7]);

/* one sublattice pass (Sec. II): color 0 = (i+j+k) even ("red"), 1 = odd.
 * acc[i] = 1/0 for cells of that color, -1 otherwise; dec[i] = decision value
 * d = dF/kT - p*ln(m'/m) + ln(u3) (accept iff d < 0); band[i] = sum of |terms|/kT.
 * Any of acc/dec/band may be NULL. Returns the number of accepted moves. */
int64_t orc_pass(orc_ctx *c, double *m, const double *H, int color, uint32_t sweep,
                 uint32_t chain, uint64_t seed, double theta_deg,
                 int8_t *acc, double *dec, double *band);

/* serial pass in index order with the demag field updated after every accepted move
 * (App. B): Eq. 14 against the current field, plus the self term when the
 * problem's demag_self is set; H is updated in place. */
int64_t orc_serial_sweep(orc_ctx *c, double *m, double *H, uint32_t sweep,
                         uint32_t chain, uint64_t seed, double theta_deg);

/* App. B (Fig. 11): mean |dF_term| / kT of the trial moves of every cell at state
 * m with frozen field H (both sublattices against the same state; the moves the
 * sweep draws at iteration `sweep`): out = [ex, dmi, an, zee, long, demag]. */
void orc_trial_terms(orc_ctx *c, const double *m, const double *H, uint32_t sweep, uint32_t chain,
                     uint64_t seed, double theta_deg, double out[6]);

/* Sec. II transverse check (Fig. 1d-f): histogram of the polar angle of every
 * cell to the mean direction of m, `bins` equal bins on [lo, hi), outside
 * angles in hist[bins]; mean_dir (optional) receives the mean direction. */
void orc_angle_hist(const orc_ctx *c, const double *m, int bins, double lo, double hi, int64_t *hist,
                    double mean_dir[3]);

/* Sec. III comparison method (SDesc): steepest descent over directions with
 * |m_i| = m_e(T_i), Barzilai-Borwein steps, until the largest normalized
 * torque is below tol (or maxit steps).  m in/out (3 n).  Returns 0 when
 * converged, 1 otherwise. */
int orc_sdesc(orc_ctx *c, double *m, int maxit, double tol, int *iters, double *torque);

/* Run state carried across orc_run calls. */
typedef struct {
    uint64_t seed;
    uint32_t chain;
    uint32_t sweep;             /* global sweep counter (Philox counter word 1) */
    double theta_deg;           /* cone half-angle */
    int64_t win_acc, win_att;   /* acceptance window counters */
    int adapt;                  /* adapt the cone angle every 100 sweeps */
    int demag_mode;             /* 0 off, 1 once per sweep, 2 before each pass, 3 serial (App. B) */
    int stripes;                /* demag_mode 2: each pass in this many bands of rows
                                   (j + ny k), the field recomputed before every band */
} orc_run_state;

/* n full sweeps; obs (may be NULL) accumulates a snapshot every obs_every sweeps */
int64_t orc_run(orc_ctx *c, double *m, int64_t n, orc_run_state *st, orc_obs *obs, int obs_every);
void    orc_obs_accumulate(const orc_ctx *c, const double *m, orc_obs *obs);
/* |m| histogram of a state in FP64: bins equal bins on [0, hmax), overflow last */
void    orc_hist(const double *m, int64_t n, int bins, double hmax, int64_t *hist);
/* cone angle adaptation rule (Sec. II) */
double  orc_adapt_theta(double theta_deg, int64_t acc, int64_t att);
/* initial state: uniform direction dir with length len, or random directions
 * from Philox counter (cell, 0, chain, 1) when random != 0 */
void    orc_init_state(const orc_ctx *c, double *m, int random, const double dir[3],
                       double len, uint32_t chain, uint64_t seed);

#ifdef __cplusplus
}
#endif
#endif
