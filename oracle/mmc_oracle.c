/*
 * mmc_oracle.c -- plain serial FP64 oracle of the micromagnetic Monte Carlo
 * method (arXiv:2106.05593).  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark are its only users.
 *
 * Written for readability against the paper, not speed: every energy change is
 * the difference of the energies of the bonds and sites that touch the cell, the
 * demag field is a direct sum or a plain radix-2 FFT convolution, and loops run
 * in index order.
 *
 * Pins (checked in tests/test_oracle_*.py, CPU only):
 *   Philox4x32-10        known-answer vectors of the published generator
 *   m_e, chi (Eq. 8-9)   T->0 and near-Tc asymptotes, closed form above Tc,
 *                        fixed-point residual
 *   energies (Eq. 10-15) pair energies equal half the per-vector sums of
 *                        Eq. 10 / Eq. 15 / Eq. 14 on periodic lattices; brute-force
 *                        dE of the local energy change; analytic gradient vs
 *                        central differences
 *   acceptance (Eq. 5)   single-cell length law = stationary law of the exact
 *                        length-move kernel; Eq. 7 within its sigma bias;
 *                        mutants with power 1 or 2 rejected
 *   cone + Zeeman        Langevin-type closed form of <m_x>
 *   Newell tensor        self term trace 1, cube 1/3, uniform-prism factors of
 *                        Aharoni's closed form; near/far formulas agree
 *   FFT demag            direct sum agreement
 *   periodic demag       exact circular-shift covariance; the thickness-averaged
 *                        field of a cosine magnetization in a film infinite in
 *                        the plane (closed form of the charge sheets, summed over
 *                        the cell aliases); half-period offsets by hand
 *   serial form (App. B) per-move field updates equal the direct sum of the final
 *                        state; without demag equal to pass-by-pass application
 *   row bands            one band = demag before each pass; without demag any
 *                        banding equals the plain iteration
 *   trial-term sizes     exchange and Zeeman means of a uniform state equal their
 *                        closed forms over the proposal (App. B, Fig. 11)
 *   SDesc (Sec. III)     Stoner-Wohlfarth angle of a single cell; torque criterion
 *   angle histogram      cap and sphere densities (Fig. 1d-f)
 *
 * Parity unpinned: equilibria of interacting chains (only GPU-oracle agreement
 * within standard errors is available).
 */
#include "mmc_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ========================================================================== */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11.  Round: two 32x32->64 multiplies of counter words 0 and 2
 * by the round multipliers, output words mixed with the round key; the key is
 * bumped by the Weyl constants between rounds.                                */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 23-bit uniform in (0,1): ((r >> 9) + 1/2) * 2^-23, exact in FP32 and FP64
 * (24 significant bits at most). */
double orc_u01(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

static void draw4(uint32_t cell, uint32_t sweep, uint32_t chain, uint32_t tag,
                  uint64_t seed, double u[4])
{
    uint32_t ctr[4] = {cell, sweep, chain, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    for (int k = 0; k < 4; ++k) u[k] = orc_u01(r[k]);
}

/* ========================================================================== */
/* Thermodynamics (Sec. II, Eqs. 7-9, 13).                                     */

/* Coefficients a_n of coth x - 1/x = sum_{n>=1} a_n x^{2n-1}: a_n = (-1)^{n+1}
 * 2 zeta(2n) / pi^{2n} (the Bernoulli-number series of coth).  zeta(2n) is
 * summed directly for n >= 5 (the tail is below 1e-17 relative). */
#define LANG_TERMS 13
static double lang_coef[LANG_TERMS];
static int lang_ready = 0;

static void lang_init(void)
{
    if (lang_ready) return;
    const double pi2 = PI * PI;
    double z[LANG_TERMS];
    z[0] = pi2 / 6.0;
    z[1] = pi2 * pi2 / 90.0;
    z[2] = pi2 * pi2 * pi2 / 945.0;
    z[3] = pi2 * pi2 * pi2 * pi2 / 9450.0;
    for (int n = 5; n <= LANG_TERMS; ++n) {
        double sum = 0.0;
        for (int k = 400; k >= 1; --k) sum += pow((double)k, -2.0 * n);
        z[n - 1] = sum;
    }
    for (int n = 1; n <= LANG_TERMS; ++n)
        lang_coef[n - 1] = ((n % 2) ? 2.0 : -2.0) * z[n - 1] / pow(PI, 2.0 * n);
    lang_ready = 1;
}

/* Langevin function B(x) = coth(x) - 1/x (Eq. 8); the series below |x| = 0.5,
 * where the difference of the two terms would cancel. */
double orc_langevin(double x)
{
    if (fabs(x) < 0.5) {
        lang_init();
        double x2 = x * x, acc = 0.0;
        for (int n = LANG_TERMS; n >= 1; --n) acc = acc * x2 + lang_coef[n - 1];
        return x * acc;
    }
    return 1.0 / tanh(x) - 1.0 / x;
}

/* B'(x) = 1/x^2 - 1/sinh^2(x); the differentiated series below |x| = 0.5. */
double orc_langevin_d(double x)
{
    double ax = fabs(x);
    if (ax < 0.5) {
        lang_init();
        double x2 = x * x, acc = 0.0;
        for (int n = LANG_TERMS; n >= 1; --n) acc = acc * x2 + (2.0 * n - 1.0) * lang_coef[n - 1];
        return acc;
    }
    if (ax > 40.0) return 1.0 / (x * x);
    double s = sinh(x);
    return 1.0 / (x * x) - 1.0 / (s * s);
}

/* Temperatures within 1 mK of Tc are evaluated 1 mK away on their own side,
 * where Eq. 8 is finite. */
static double tc_guard(double T, double Tc)
{
    if (fabs(T - Tc) < 1e-3) return (T < Tc) ? Tc - 1e-3 : Tc + 1e-3;
    return T;
}

/* Eq. 9 with zero field: m_e = B(m_e * 3Tc/T).  Below Tc the positive root is
 * bracketed in (0, 1] and found by bisection; m_e = 0 at and above Tc. */
double orc_me(double T, double Tc)
{
    T = tc_guard(T, Tc);
    if (T >= Tc) return 0.0;
    double b = 3.0 * Tc / T;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        double g = orc_langevin(b * mid) - mid;
        if (g > 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Eq. 8: chi = (mu/(kB T)) B'(x) / (1 - B'(x) 3Tc/T), x = m_e 3Tc/T  (1/T). */
double orc_chi(double T, double Tc, double mu)
{
    T = tc_guard(T, Tc);
    double me = orc_me(T, Tc);
    double x = me * 3.0 * Tc / T;
    double bp = orc_langevin_d(x);
    return (mu / (ORC_KB * T)) * bp / (1.0 - bp * 3.0 * Tc / T);
}

/* Eq. 13 with the cap; the cap is used at and above Tc. */
double orc_sigma(double T, double Tc, double mu, double V, double Ms0, double cap)
{
    T = tc_guard(T, Tc);
    if (T >= Tc) return cap;
    double me = orc_me(T, Tc);
    double s = 2.0 * me * sqrt(orc_chi(T, Tc, mu) * ORC_KB * T / (V * Ms0));
    return s < cap ? s : cap;
}

/* Exponent of Eq. 7 times kT, given m_e(T) and chi(T): the longitudinal free
 * energy of one cell (J). */
static double long_energy_tab(double m, double me, double chi, double T, double Tc,
                              double V, double Ms0)
{
    T = tc_guard(T, Tc);
    if (T < Tc) {
        double d = m * m - me * me;
        return V * Ms0 * d * d / (8.0 * chi * me * me);
    }
    return V * Ms0 * m * m / (2.0 * chi) * (1.0 + 3.0 * Tc * m * m / (10.0 * (T - Tc)));
}

double orc_long_energy(double m, double T, double Tc, double mu, double V, double Ms0)
{
    return long_energy_tab(m, orc_me(T, Tc), orc_chi(T, Tc, mu), T, Tc, V, Ms0);
}

/* ========================================================================== */
/* Demagnetizing tensor (Sec. III, Eq. 14).  N(R) is the field in a target cell,
 * averaged over it, from a uniformly magnetized source cell at offset R:
 * H = -N M.  Near field: Newell, Williams & Dunlop (1993) f and g functions
 * with the 27-point second difference, in long double.  Far field: the same
 * cell-pair average of the point-dipole kernel, by Gauss-Legendre quadrature
 * over the triangular distribution of the difference of two uniform points. */

static long double nf(long double x, long double y, long double z)
{
    x = fabsl(x); y = fabsl(y); z = fabsl(z);
    long double x2 = x * x, y2 = y * y, z2 = z * z;
    long double R = sqrtl(x2 + y2 + z2);
    if (R == 0.0L) return 0.0L;
    long double r = 0.0L;
    if (y > 0 && x2 + z2 > 0) r += 0.5L * y * (z2 - x2) * asinhl(y / sqrtl(x2 + z2));
    if (z > 0 && x2 + y2 > 0) r += 0.5L * z * (y2 - x2) * asinhl(z / sqrtl(x2 + y2));
    if (x > 0 && y > 0 && z > 0) r -= x * y * z * atanl(y * z / (x * R));
    r += (2.0L * x2 - y2 - z2) * R / 6.0L;
    return r;
}

static long double ng(long double x, long double y, long double z)
{
    int s = 1;
    if (x < 0) { x = -x; s = -s; }
    if (y < 0) { y = -y; s = -s; }
    z = fabsl(z);
    if (x == 0.0L || y == 0.0L) return 0.0L;
    long double x2 = x * x, y2 = y * y, z2 = z * z;
    long double R = sqrtl(x2 + y2 + z2);
    long double r = 0.0L;
    if (z > 0) r += x * y * z * asinhl(z / sqrtl(x2 + y2));
    r += y / 6.0L * (3.0L * z2 - y2) * asinhl(x / sqrtl(y2 + z2));
    r += x / 6.0L * (3.0L * z2 - x2) * asinhl(y / sqrtl(x2 + z2));
    if (z > 0) {
        r -= z2 * z / 6.0L * atanl(x * y / (z * R));
        r -= z * y2 / 2.0L * atanl(x * z / (y * R));
        r -= z * x2 / 2.0L * atanl(y * z / (x * R));
    }
    r -= x * y * R / 3.0L;
    return s * r;
}

/* sum over e in {-1,0,1}^3 of w(ex)w(ey)w(ez) F(X+ex dx, ...), w(0)=2, w(+-1)=-1 */
static long double d27(long double (*F)(long double, long double, long double),
                       long double X, long double Y, long double Z,
                       long double dx, long double dy, long double dz)
{
    static const long double w[3] = {-1.0L, 2.0L, -1.0L};
    long double acc = 0.0L;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c)
                acc += w[a + 1] * w[b + 1] * w[c + 1] *
                       F(X + a * dx, Y + b * dy, Z + c * dz);
    return acc;
}

/* out = {xx, yy, zz, xy, xz, yz} */
void orc_newell(double dx, double dy, double dz, double X, double Y, double Z, double out[6])
{
    long double V4pi = 4.0L * (long double)PI * (long double)dx * dy * dz;
    long double lx = X, ly = Y, lz = Z, ldx = dx, ldy = dy, ldz = dz;
    /* Nxx uses f(x,y,z); Nyy f(y,x,z); Nzz f(z,y,x); Nxy g(x,y,z); Nxz g(x,z,y); Nyz g(y,z,x) */
    out[0] = (double)(d27(nf, lx, ly, lz, ldx, ldy, ldz) / V4pi);
    out[1] = (double)(d27(nf, ly, lx, lz, ldy, ldx, ldz) / V4pi);
    out[2] = (double)(d27(nf, lz, ly, lx, ldz, ldy, ldx) / V4pi);
    out[3] = (double)(d27(ng, lx, ly, lz, ldx, ldy, ldz) / V4pi);
    out[4] = (double)(d27(ng, lx, lz, ly, ldx, ldz, ldy) / V4pi);
    out[5] = (double)(d27(ng, ly, lz, lx, ldy, ldz, ldx) / V4pi);
}

/* Gauss-Legendre nodes/weights on [-1,1], n <= 8, by Newton on P_n. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double t = cos(PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* nodes and weights of the triangular density (d-|u|)/d^2 on [-d,d], using an
 * npts-point Gauss-Legendre rule on each half */
static int tri_rule(double d, int npts, double *u, double *w)
{
    double gx[16], gw[16];
    gauss_legendre(npts, gx, gw);
    int k = 0;
    for (int half = 0; half < 2; ++half)
        for (int i = 0; i < npts; ++i) {
            double t = 0.5 * d * (gx[i] + 1.0);             /* in [0, d] */
            double uu = half ? t : -t;
            u[k] = uu;
            w[k] = 0.5 * d * gw[i] * (d - t) / (d * d);
            ++k;
        }
    return k;
}

/* N_ab(R) = -(V/4pi) E_u[(3 r_a r_b - delta_ab r^2)/r^5], r = R + u */
void orc_tensor_quad(double dx, double dy, double dz, double X, double Y, double Z,
                     int npts, double out[6])
{
    double ux[32], wx[32], uy[32], wy[32], uz[32], wz[32];
    int nxq = tri_rule(dx, npts, ux, wx);
    int nyq = tri_rule(dy, npts, uy, wy);
    int nzq = tri_rule(dz, npts, uz, wz);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < nxq; ++a)
        for (int b = 0; b < nyq; ++b)
            for (int c = 0; c < nzq; ++c) {
                double rx = X + ux[a], ry = Y + uy[b], rz = Z + uz[c];
                double r2 = rx * rx + ry * ry + rz * rz;
                double r = sqrt(r2);
                double i5 = 1.0 / (r2 * r2 * r);
                double w = wx[a] * wy[b] * wz[c];
                acc[0] += w * (3.0 * rx * rx - r2) * i5;
                acc[1] += w * (3.0 * ry * ry - r2) * i5;
                acc[2] += w * (3.0 * rz * rz - r2) * i5;
                acc[3] += w * (3.0 * rx * ry) * i5;
                acc[4] += w * (3.0 * rx * rz) * i5;
                acc[5] += w * (3.0 * ry * rz) * i5;
            }
    double V = dx * dy * dz;
    for (int k = 0; k < 6; ++k) out[k] = -V / (4.0 * PI) * acc[k];
}

/* Newell below 20 h_max (Euclidean), where its cancellation in long double stays
 * below ~1e-10 relative; the 5-point-per-half quadrature beyond, where its error
 * ~ (h/R)^10 is below 1e-13. */
void orc_tensor(double dx, double dy, double dz, double X, double Y, double Z, double out[6])
{
    double hmax = dx > dy ? dx : dy;
    if (dz > hmax) hmax = dz;
    double R = sqrt(X * X + Y * Y + Z * Z);
    if (R < 20.0 * hmax) orc_newell(dx, dy, dz, X, Y, Z, out);
    else orc_tensor_quad(dx, dy, dz, X, Y, Z, 5, out);
}

/* ========================================================================== */
/* Context                                                                     */

struct orc_ctx {
    orc_problem p;
    int n;                                  /* ncell */
    double V;
    double *Ms0, *K1, *K2, *eA, *Tc, *T;    /* copies */
    int *grain;
    double *me, *chi, *sigma, *K1T, *K2T, *kT;
    /* demag tensor on offsets o in [-(n-1), n-1] per axis, 6 comps */
    int ox, oy, oz;                         /* n-1 per axis */
    double *Nt;
    /* FFT convolution */
    int Px, Py, Pz;
    double complex *Nhat;                   /* 6 * P */
    double complex *work;                   /* 3 * P */
};

int orc_ncell(const orc_ctx *c) { return c->n; }

static int pow2_at_least(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

static double *dup_d(const double *src, int n, double dflt)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) d[i] = src ? src[i] : dflt;
    return d;
}

static size_t toff(const orc_ctx *c, int X, int Y, int Z)
{
    int wx = 2 * c->ox + 1, wy = 2 * c->oy + 1;
    return (size_t)(X + c->ox) + (size_t)wx * ((size_t)(Y + c->oy) + (size_t)wy * (size_t)(Z + c->oz));
}

static void fft1(double complex *a, int n, int stride, int inverse);

/* Demag kernel of Eq. 14 at cell offset (X, Y, Z).  Open axes: the tensor at
 * that offset.  The granular and chiral films of Sec. III-IV are periodic in the
 * plane; the paper does not spell out the periodic convolution, and the reading
 * taken here is the lattice sum over periodic
 * images truncated at P = demag_images images on each side of the mesh: along a
 * periodic axis of extent n an offset X stands for the displacements
 * X~ + p n, p = -P..P, with X~ the minimal image of X (|X~| <= n/2); when X~ is
 * exactly half the period both minimal images n/2 and -n/2 are taken, with weight
 * 1/2 each, so that the kernel keeps the parity of the tensor. */
void orc_kernel(const orc_ctx *c, int X, int Y, int Z, double out[6])
{
    const orc_problem *p = &c->p;
    const int n[3] = {p->nx, p->ny, p->nz}, o[3] = {X, Y, Z};
    int nrep[3], rep[3][2], P[3];
    double wrep[3][2];
    for (int a = 0; a < 3; ++a) {
        if (p->demag_images <= 0 || !p->pbc[a]) {
            nrep[a] = 1; rep[a][0] = o[a]; wrep[a][0] = 1.0; P[a] = 0;
            continue;
        }
        P[a] = p->demag_images;
        int r = ((o[a] % n[a]) + n[a]) % n[a];          /* X mod n in [0, n) */
        if (2 * r == n[a]) {
            nrep[a] = 2;
            rep[a][0] = r; rep[a][1] = r - n[a];
            wrep[a][0] = wrep[a][1] = 0.5;
        } else {
            nrep[a] = 1;
            rep[a][0] = 2 * r < n[a] ? r : r - n[a];
            wrep[a][0] = 1.0;
        }
    }
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    for (int ra = 0; ra < nrep[0]; ++ra)
        for (int rb = 0; rb < nrep[1]; ++rb)
            for (int rc = 0; rc < nrep[2]; ++rc) {
                double w = wrep[0][ra] * wrep[1][rb] * wrep[2][rc];
                for (int pz = -P[2]; pz <= P[2]; ++pz)
                    for (int py = -P[1]; py <= P[1]; ++py)
                        for (int px = -P[0]; px <= P[0]; ++px) {
                            double t[6];
                            int dx = rep[0][ra] + px * n[0];
                            int dy = rep[1][rb] + py * n[1];
                            int dz = rep[2][rc] + pz * n[2];
                            orc_tensor(p->h[0], p->h[1], p->h[2], dx * p->h[0], dy * p->h[1], dz * p->h[2], t);
                            for (int k = 0; k < 6; ++k) out[k] += w * t[k];
                        }
            }
}

static void build_demag(orc_ctx *c)
{
    const orc_problem *p = &c->p;
    c->ox = p->nx - 1; c->oy = p->ny - 1; c->oz = p->nz - 1;
    size_t nt = (size_t)(2 * c->ox + 1) * (2 * c->oy + 1) * (2 * c->oz + 1);
    c->Nt = (double *)malloc(sizeof(double) * 6 * nt);
    /* compute one octant, fill the rest by parity: xx,yy,zz even; xy odd in x,y;
     * xz odd in x,z; yz odd in y,z (the periodic kernel has the same parity).
     * The convolution below is linear over offsets -(n-1)..n-1, which with the
     * periodic kernel K(X) = K(X mod n) is the circular convolution exactly. */
    for (int Z = 0; Z <= c->oz; ++Z)
        for (int Y = 0; Y <= c->oy; ++Y)
            for (int X = 0; X <= c->ox; ++X) {
                double t[6];
                orc_kernel(c, X, Y, Z, t);
                for (int sz = -1; sz <= 1; sz += 2)
                    for (int sy = -1; sy <= 1; sy += 2)
                        for (int sx = -1; sx <= 1; sx += 2) {
                            if ((X == 0 && sx < 0) || (Y == 0 && sy < 0) || (Z == 0 && sz < 0)) continue;
                            double *o = c->Nt + 6 * toff(c, sx * X, sy * Y, sz * Z);
                            o[0] = t[0]; o[1] = t[1]; o[2] = t[2];
                            o[3] = sx * sy * t[3];
                            o[4] = sx * sz * t[4];
                            o[5] = sy * sz * t[5];
                        }
            }
    /* padded kernel spectra for the FFT path */
    c->Px = p->nx > 1 ? pow2_at_least(2 * p->nx) : 1;
    c->Py = p->ny > 1 ? pow2_at_least(2 * p->ny) : 1;
    c->Pz = p->nz > 1 ? pow2_at_least(2 * p->nz) : 1;
    size_t P = (size_t)c->Px * c->Py * c->Pz;
    c->Nhat = (double complex *)calloc(6 * P, sizeof(double complex));
    c->work = (double complex *)calloc(3 * P, sizeof(double complex));
    for (int Z = -c->oz; Z <= c->oz; ++Z)
        for (int Y = -c->oy; Y <= c->oy; ++Y)
            for (int X = -c->ox; X <= c->ox; ++X) {
                int ix = (X + c->Px) % c->Px, iy = (Y + c->Py) % c->Py, iz = (Z + c->Pz) % c->Pz;
                size_t q = (size_t)ix + (size_t)c->Px * ((size_t)iy + (size_t)c->Py * iz);
                const double *t = c->Nt + 6 * toff(c, X, Y, Z);
                for (int k = 0; k < 6; ++k) c->Nhat[k * P + q] = t[k];
            }
    for (int k = 0; k < 6; ++k) {
        double complex *a = c->Nhat + k * P;
        for (int z = 0; z < c->Pz; ++z)
            for (int y = 0; y < c->Py; ++y) fft1(a + (size_t)c->Px * (y + (size_t)c->Py * z), c->Px, 1, 0);
        for (int z = 0; z < c->Pz; ++z)
            for (int x = 0; x < c->Px; ++x) fft1(a + x + (size_t)c->Px * c->Py * z, c->Py, c->Px, 0);
        for (int y = 0; y < c->Py; ++y)
            for (int x = 0; x < c->Px; ++x) fft1(a + x + (size_t)c->Px * y, c->Pz, c->Px * c->Py, 0);
    }
}

static void compute_tables(orc_ctx *c)
{
    const orc_problem *p = &c->p;
    int l1 = p->aniso_cubic ? 10 : 3;       /* m_e^{l(l+1)/2}: l = 2 (uniaxial K1), 4 */
    int l2 = p->aniso_cubic ? 21 : 10;      /* l = 4 (uniaxial K2), 6 (cubic K2) */
    for (int i = 0; i < c->n; ++i) {
        double T = c->T[i], Tc = c->Tc[i];
        c->me[i] = orc_me(T, Tc);
        c->chi[i] = orc_chi(T, Tc, p->mu);
        c->sigma[i] = orc_sigma(T, Tc, p->mu, c->V, c->Ms0[i], p->sigma_cap);
        c->K1T[i] = c->K1[i] * pow(c->me[i], l1);
        c->K2T[i] = c->K2[i] * pow(c->me[i], l2);
        c->kT[i] = ORC_KB * T;
    }
}

orc_ctx *orc_create(const orc_problem *p)
{
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->p = *p;
    c->n = p->nx * p->ny * p->nz;
    c->V = p->h[0] * p->h[1] * p->h[2];
    if (c->p.len_power == 0) c->p.len_power = 4;
    int n = c->n;
    c->Ms0 = dup_d(p->Ms0, n, 0.0);
    c->K1 = dup_d(p->K1, n, 0.0);
    c->K2 = dup_d(p->K2, n, 0.0);
    c->Tc = dup_d(p->Tc, n, 0.0);
    c->T = dup_d(p->T, n, 0.0);
    /* e_A is the symmetry-axis direction of Eq. 11: stored as a unit vector */
    c->eA = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    for (int i = 0; i < 3 * n; ++i) c->eA[i] = p->eA ? p->eA[i] : (i % 3 == 2 ? 1.0 : 0.0);
    for (int i = 0; i < n; ++i) {
        double *e = c->eA + 3 * i;
        double l = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        if (l > 0.0) { e[0] /= l; e[1] /= l; e[2] /= l; }
        else { e[0] = 0.0; e[1] = 0.0; e[2] = 1.0; }
    }
    c->grain = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) c->grain[i] = p->grain ? p->grain[i] : 0;
    c->p.Ms0 = c->p.K1 = c->p.K2 = c->p.eA = c->p.Tc = c->p.T = NULL;
    c->p.grain = NULL;
    c->me = dup_d(NULL, n, 0); c->chi = dup_d(NULL, n, 0); c->sigma = dup_d(NULL, n, 0);
    c->K1T = dup_d(NULL, n, 0); c->K2T = dup_d(NULL, n, 0); c->kT = dup_d(NULL, n, 0);
    compute_tables(c);
    if (p->demag) build_demag(c);
    return c;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->Ms0); free(c->K1); free(c->K2); free(c->eA); free(c->Tc); free(c->T);
    free(c->grain); free(c->me); free(c->chi); free(c->sigma); free(c->K1T);
    free(c->K2T); free(c->kT); free(c->Nt); free(c->Nhat); free(c->work);
    free(c);
}

void orc_set_field(orc_ctx *c, const double B[3])
{
    c->p.B[0] = B[0]; c->p.B[1] = B[1]; c->p.B[2] = B[2];
}

void orc_tables(const orc_ctx *c, double *me, double *chi, double *sigma, double *K1T, double *K2T)
{
    for (int i = 0; i < c->n; ++i) {
        if (me) me[i] = c->me[i];
        if (chi) chi[i] = c->chi[i];
        if (sigma) sigma[i] = c->sigma[i];
        if (K1T) K1T[i] = c->K1T[i];
        if (K2T) K2T[i] = c->K2T[i];
    }
}

/* ========================================================================== */
/* Demag field                                                                 */

/* iterative radix-2 complex FFT of n (power of 2) points with stride; forward
 * uses exp(-2 pi i k j / n); the inverse is unnormalized */
static void fft1(double complex *a, int n, int stride, int inverse)
{
    if (n <= 1) return;
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double complex t = a[(size_t)i * stride];
            a[(size_t)i * stride] = a[(size_t)j * stride];
            a[(size_t)j * stride] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        double ang = 2.0 * PI / len * (inverse ? 1.0 : -1.0);
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                double complex w = cos(ang * k) + I * sin(ang * k);
                double complex u = a[(size_t)(i + k) * stride];
                double complex v = a[(size_t)(i + k + len / 2) * stride] * w;
                a[(size_t)(i + k) * stride] = u + v;
                a[(size_t)(i + k + len / 2) * stride] = u - v;
            }
    }
}

static void fft3(orc_ctx *c, double complex *a, int inverse)
{
    int Px = c->Px, Py = c->Py, Pz = c->Pz;
    for (int z = 0; z < Pz; ++z)
        for (int y = 0; y < Py; ++y) fft1(a + (size_t)Px * (y + (size_t)Py * z), Px, 1, inverse);
    for (int z = 0; z < Pz; ++z)
        for (int x = 0; x < Px; ++x) fft1(a + x + (size_t)Px * Py * z, Py, Px, inverse);
    for (int y = 0; y < Py; ++y)
        for (int x = 0; x < Px; ++x) fft1(a + x + (size_t)Px * y, Pz, Px * Py, inverse);
}

/* Eq. 14: H_i = -sum_j N(r_i - r_j) Ms0_j m_j */
void orc_demag_field(orc_ctx *c, const double *m, double *H, int method)
{
    const orc_problem *p = &c->p;
    int nx = p->nx, ny = p->ny, nz = p->nz;
    if (!p->demag) { memset(H, 0, sizeof(double) * 3 * (size_t)c->n); return; }
    if (method == 0) {
        for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
            double h[3] = {0, 0, 0};
            for (int kk = 0; kk < nz; ++kk) for (int jj = 0; jj < ny; ++jj) for (int ii = 0; ii < nx; ++ii) {
                int q = ii + nx * (jj + ny * kk);
                const double *t = c->Nt + 6 * toff(c, i - ii, j - jj, k - kk);
                double Mx = c->Ms0[q] * m[3 * q], My = c->Ms0[q] * m[3 * q + 1], Mz = c->Ms0[q] * m[3 * q + 2];
                h[0] -= t[0] * Mx + t[3] * My + t[4] * Mz;
                h[1] -= t[3] * Mx + t[1] * My + t[5] * Mz;
                h[2] -= t[4] * Mx + t[5] * My + t[2] * Mz;
            }
            int q = i + nx * (j + ny * k);
            H[3 * q] = h[0]; H[3 * q + 1] = h[1]; H[3 * q + 2] = h[2];
        }
        return;
    }
    size_t P = (size_t)c->Px * c->Py * c->Pz;
    double complex *w = c->work;
    memset(w, 0, sizeof(double complex) * 3 * P);
    for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
        int q = i + nx * (j + ny * k);
        size_t s = (size_t)i + (size_t)c->Px * ((size_t)j + (size_t)c->Py * k);
        for (int a = 0; a < 3; ++a) w[a * P + s] = c->Ms0[q] * m[3 * q + a];
    }
    for (int a = 0; a < 3; ++a) fft3(c, w + a * P, 0);
    for (size_t s = 0; s < P; ++s) {
        double complex Mx = w[s], My = w[P + s], Mz = w[2 * P + s];
        double complex *N = c->Nhat;
        double complex hx = -(N[s] * Mx + N[3 * P + s] * My + N[4 * P + s] * Mz);
        double complex hy = -(N[3 * P + s] * Mx + N[P + s] * My + N[5 * P + s] * Mz);
        double complex hz = -(N[4 * P + s] * Mx + N[5 * P + s] * My + N[2 * P + s] * Mz);
        w[s] = hx; w[P + s] = hy; w[2 * P + s] = hz;
    }
    for (int a = 0; a < 3; ++a) fft3(c, w + a * P, 1);
    double inv = 1.0 / (double)P;
    for (int k = 0; k < nz; ++k) for (int j = 0; j < ny; ++j) for (int i = 0; i < nx; ++i) {
        int q = i + nx * (j + ny * k);
        size_t s = (size_t)i + (size_t)c->Px * ((size_t)j + (size_t)c->Py * k);
        for (int a = 0; a < 3; ++a) H[3 * q + a] = creal(w[a * P + s]) * inv;
    }
}

/* ========================================================================== */
/* Energies (Eqs. 7, 10-12, 14, 15).                                           */

/* neighbour of cell (i,j,k) along axis a, direction dir (+1/-1); -1 if absent */
static int neighbour(const orc_ctx *c, int i, int j, int k, int a, int dir)
{
    const orc_problem *p = &c->p;
    int v[3] = {i, j, k};
    int n[3] = {p->nx, p->ny, p->nz};
    v[a] += dir;
    if (v[a] < 0 || v[a] >= n[a]) {
        if (!p->pbc[a]) return -1;
        v[a] = (v[a] + n[a]) % n[a];
    }
    return v[0] + p->nx * (v[1] + p->ny * v[2]);
}

static double bond_scale(const orc_ctx *c, int q, int r)
{
    return c->grain[q] == c->grain[r] ? 1.0 : c->p.grain_exch_scale;
}

/* exchange energy of the bond (q, r) along axis a: c_ex |m_q - m_r|^2,
 * c_ex = V A0 / h_a^2 (Eq. 10 summed over vectors counts each bond twice) */
static double bond_ex(const orc_ctx *c, const double *mq, const double *mr, int a, double s)
{
    double h = c->p.h[a];
    double cex = c->V * c->p.A0 / (h * h);
    double dx = mq[0] - mr[0], dy = mq[1] - mr[1], dz = mq[2] - mr[2];
    return s * cex * (dx * dx + dy * dy + dz * dz);
}

/* interfacial DMI energy of the bond q -> r = q + e_a (a = 0, 1):
 * -(V D0 / h_a) d.(m_q x m_r), d = z x e_a (Eq. 15 with central differences,
 * summed over vectors, counts each bond twice) */
static double bond_dmi(const orc_ctx *c, const double *mq, const double *mr, int a, double s)
{
    if (a == 2) return 0.0;
    double cd = c->V * c->p.D0 / c->p.h[a];
    double cross_x = mq[1] * mr[2] - mq[2] * mr[1];
    double cross_y = mq[2] * mr[0] - mq[0] * mr[2];
    /* z x x = y ; z x y = -x */
    double dcross = (a == 0) ? cross_y : -cross_x;
    return -s * cd * dcross;
}

/* single-site anisotropy (Eq. 11 uniaxial or Eq. 12 cubic), V on both terms,
 * direction from the unit vector m/|m| */
static double site_anis(const orc_ctx *c, int q, const double *m)
{
    double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    if (len == 0.0) return 0.0;
    double ux = m[0] / len, uy = m[1] / len, uz = m[2] / len;
    if (c->p.aniso_cubic) {
        double a2 = ux * ux, b2 = uy * uy, g2 = uz * uz;
        return c->V * (c->K1T[q] * (a2 * b2 + a2 * g2 + b2 * g2) + c->K2T[q] * a2 * b2 * g2);
    }
    const double *e = c->eA + 3 * q;
    double d = ux * e[0] + uy * e[1] + uz * e[2];
    double s = 1.0 - d * d;
    return c->V * (c->K1T[q] * s + c->K2T[q] * s * s);
}

/* Zeeman: -mu0 V M.H = -V Ms0 m.B */
static double site_zee(const orc_ctx *c, int q, const double *m)
{
    const double *B = c->p.B;
    return -c->V * c->Ms0[q] * (m[0] * B[0] + m[1] * B[1] + m[2] * B[2]);
}

static double site_long(const orc_ctx *c, int q, const double *m)
{
    double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    return long_energy_tab(len, c->me[q], c->chi[q], c->T[q], c->Tc[q], c->V, c->Ms0[q]);
}

void orc_energy(orc_ctx *c, const double *m, double out[7])
{
    const orc_problem *p = &c->p;
    double ex = 0, dmi = 0, an = 0, ze = 0, lo = 0, de = 0;
    for (int k = 0; k < p->nz; ++k) for (int j = 0; j < p->ny; ++j) for (int i = 0; i < p->nx; ++i) {
        int q = i + p->nx * (j + p->ny * k);
        const double *mq = m + 3 * q;
        for (int a = 0; a < 3; ++a) {
            int r = neighbour(c, i, j, k, a, +1);
            if (r < 0) continue;
            double s = bond_scale(c, q, r);
            ex += bond_ex(c, mq, m + 3 * r, a, s);
            dmi += bond_dmi(c, mq, m + 3 * r, a, s);
        }
        an += site_anis(c, q, mq);
        ze += site_zee(c, q, mq);
        lo += site_long(c, q, mq);
    }
    if (p->demag) {
        double *H = (double *)malloc(sizeof(double) * 3 * (size_t)c->n);
        orc_demag_field(c, m, H, c->n <= 4096 ? 0 : 1);
        for (int q = 0; q < c->n; ++q)
            de += -0.5 * ORC_MU0 * c->V * c->Ms0[q] *
                  (m[3 * q] * H[3 * q] + m[3 * q + 1] * H[3 * q + 1] + m[3 * q + 2] * H[3 * q + 2]);
        free(H);
    }
    out[1] = ex; out[2] = dmi; out[3] = an; out[4] = ze; out[5] = lo; out[6] = de;
    out[0] = ex + dmi + an + ze + lo + de;
}

/* Sum over vectors of the per-vector free energies as the paper writes them:
 * Eq. 10 with the discrete Laplacian, Eq. 15 with central differences, Eq. 14.
 * On periodic lattices (and with the demag term always) each equals twice the
 * corresponding energy. */
void orc_pervector_sums(orc_ctx *c, const double *m, double out[3])
{
    const orc_problem *p = &c->p;
    double ex = 0, dmi = 0, de = 0;
    for (int k = 0; k < p->nz; ++k) for (int j = 0; j < p->ny; ++j) for (int i = 0; i < p->nx; ++i) {
        int q = i + p->nx * (j + p->ny * k);
        const double *mq = m + 3 * q;
        double lap[3] = {0, 0, 0};
        double divm = 0, gmz[2] = {0, 0};
        for (int a = 0; a < 3; ++a) {
            int rp = neighbour(c, i, j, k, a, +1), rm = neighbour(c, i, j, k, a, -1);
            double h = p->h[a];
            const double *mp = rp >= 0 ? m + 3 * rp : mq;    /* open edge: zero difference */
            const double *mm = rm >= 0 ? m + 3 * rm : mq;
            for (int b = 0; b < 3; ++b) lap[b] += (mp[b] + mm[b] - 2.0 * mq[b]) / (h * h);
            if (a < 2) {
                divm += (mp[a] - mm[a]) / (2.0 * h);
                gmz[a] = (mp[2] - mm[2]) / (2.0 * h);
            }
        }
        /* Eq. 10: F_ex = -V (2A/Me^2) M.lap M = -2 V A0 m.lap m */
        ex += -2.0 * c->V * p->A0 * (mq[0] * lap[0] + mq[1] * lap[1] + mq[2] * lap[2]);
        /* Eq. 15: F = -V (2D/Me^2) M.(z div M - grad Mz) = -2 V D0 m.(z div m - grad mz) */
        dmi += -2.0 * c->V * p->D0 * (mq[2] * divm - mq[0] * gmz[0] - mq[1] * gmz[1]);
    }
    if (p->demag) {
        double *H = (double *)malloc(sizeof(double) * 3 * (size_t)c->n);
        orc_demag_field(c, m, H, c->n <= 4096 ? 0 : 1);
        for (int q = 0; q < c->n; ++q)   /* Eq. 14: F_d,i = -V mu0 M_i.H_d,i */
            de += -ORC_MU0 * c->V * c->Ms0[q] *
                  (m[3 * q] * H[3 * q] + m[3 * q + 1] * H[3 * q + 1] + m[3 * q + 2] * H[3 * q + 2]);
        free(H);
    }
    out[0] = ex; out[1] = dmi; out[2] = de;
}

/* energies of all bonds touching cell q plus its site terms, with m_q = mq */
static void local_energy(const orc_ctx *c, const double *m, int q, const double *mq, double t[5])
{
    const orc_problem *p = &c->p;
    int i = q % p->nx, j = (q / p->nx) % p->ny, k = q / (p->nx * p->ny);
    double ex = 0, dmi = 0;
    for (int a = 0; a < 3; ++a) {
        int rp = neighbour(c, i, j, k, a, +1);      /* bond q -> rp */
        if (rp >= 0) {
            double s = bond_scale(c, q, rp);
            const double *mr = (rp == q) ? mq : m + 3 * rp;
            ex += bond_ex(c, mq, mr, a, s);
            dmi += bond_dmi(c, mq, mr, a, s);
        }
        int rm = neighbour(c, i, j, k, a, -1);      /* bond rm -> q */
        if (rm >= 0) {
            double s = bond_scale(c, rm, q);
            const double *mr = (rm == q) ? mq : m + 3 * rm;
            ex += bond_ex(c, mr, mq, a, s);
            dmi += bond_dmi(c, mr, mq, a, s);
        }
    }
    t[0] = ex; t[1] = dmi;
    t[2] = site_anis(c, q, mq);
    t[3] = site_zee(c, q, mq);
    t[4] = site_long(c, q, mq);
}

/* self demag tensor of one cell: offset 0 */
static const double *self_tensor(const orc_ctx *c) { return c->Nt + 6 * toff(c, 0, 0, 0); }

void orc_local_dF(orc_ctx *c, const double *m, const double *H, int q, const double mnew[3], double out[7])
{
    double a[5], b[5];
    local_energy(c, m, q, m + 3 * q, a);
    local_energy(c, m, q, mnew, b);
    double dd = 0.0;
    if (c->p.demag && H) {
        /* Eq. 14 with the field frozen: dF_d = -V mu0 dM.H_d */
        double dm[3] = {mnew[0] - m[3 * q], mnew[1] - m[3 * q + 1], mnew[2] - m[3 * q + 2]};
        double Ms = c->Ms0[q];
        dd = -ORC_MU0 * c->V * Ms * (dm[0] * H[3 * q] + dm[1] * H[3 * q + 1] + dm[2] * H[3 * q + 2]);
        if (c->p.demag_self) {
            const double *t = self_tensor(c);
            double Nd[3] = {t[0] * dm[0] + t[3] * dm[1] + t[4] * dm[2],
                            t[3] * dm[0] + t[1] * dm[1] + t[5] * dm[2],
                            t[4] * dm[0] + t[5] * dm[1] + t[2] * dm[2]};
            dd += 0.5 * ORC_MU0 * c->V * Ms * Ms * (dm[0] * Nd[0] + dm[1] * Nd[1] + dm[2] * Nd[2]);
        }
    }
    double tot = dd;
    for (int k = 0; k < 5; ++k) { out[k + 1] = b[k] - a[k]; tot += out[k + 1]; }
    out[6] = dd;
    out[0] = tot;
}

/* ========================================================================== */
/* Trial move (Sec. II): rotation uniform on the spherical cap of half-angle
 * theta around m/|m|, then |m| multiplied by a factor uniform in
 * [1 - sigma, 1 + sigma].  The basis (e1, e2) orthogonal to the direction is the
 * branchless construction of Duff et al., JCGT 6(1), 2017.                    */
static void propose(const double *m, double cos_tc, double sigma, const double u[4], double out[3])
{
    double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    double nx = m[0] / len, ny = m[1] / len, nz = m[2] / len;
    double sgn = nz >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sgn + nz);
    double b = nx * ny * a;
    double e1[3] = {1.0 + sgn * nx * nx * a, sgn * b, -sgn * nx};
    double e2[3] = {b, sgn + ny * ny * a, -ny};
    double t = u[0] * (1.0 - cos_tc);               /* 1 - cos(theta) */
    double ct = 1.0 - t;
    double st = sqrt(t * (2.0 - t));
    double phi = 2.0 * PI * u[1];
    double cp = cos(phi), sp = sin(phi);
    double s = 1.0 - sigma + 2.0 * sigma * u[2];    /* length factor */
    double newlen = len * s;
    out[0] = newlen * (ct * nx + st * (cp * e1[0] + sp * e2[0]));
    out[1] = newlen * (ct * ny + st * (cp * e1[1] + sp * e2[1]));
    out[2] = newlen * (ct * nz + st * (cp * e1[2] + sp * e2[2]));
}

static int cell_color(const orc_ctx *c, int q)
{
    const orc_problem *p = &c->p;
    int i = q % p->nx, j = (q / p->nx) % p->ny, k = q / (p->nx * p->ny);
    return (i + j + k) & 1;
}

/* Eq. 5: accept with probability min{1, (m_B/m_A)^4 exp(-dF/kT)}, i.e. iff
 * d = dF/kT - 4 ln(m_B/m_A) + ln u3 < 0 */
static int trial(orc_ctx *c, double *m, const double *H, int q, uint32_t sweep, uint32_t chain,
                 uint64_t seed, double cos_tc, double *dec, double *band)
{
    double u[4], mn[3], t[7];
    draw4((uint32_t)q + c->p.cell_base, sweep, chain, 0u, seed, u);
    propose(m + 3 * q, cos_tc, c->sigma[q], u, mn);
    orc_local_dF(c, m, H, q, mn, t);
    double kT = c->kT[q];
    double s = 1.0 - c->sigma[q] + 2.0 * c->sigma[q] * u[2];
    double d = t[0] / kT - (double)c->p.len_power * log(s) + log(u[3]);
    if (dec) *dec = d;
    if (band) {
        double sum = 0.0;
        for (int k = 1; k < 7; ++k) sum += fabs(t[k]);
        *band = sum / kT + fabs((double)c->p.len_power * log(s)) + fabs(log(u[3]));
    }
    if (d < 0.0) {
        m[3 * q] = mn[0]; m[3 * q + 1] = mn[1]; m[3 * q + 2] = mn[2];
        return 1;
    }
    return 0;
}

/* the cells of one colour in rows r0 <= j + ny k < r1 (a whole pass: 0, ny nz) */
static int64_t pass_rows(orc_ctx *c, double *m, const double *H, int color, int r0, int r1, uint32_t sweep,
                         uint32_t chain, uint64_t seed, double theta_deg,
                         int8_t *acc, double *dec, double *band)
{
    double cos_tc = cos(theta_deg * PI / 180.0);
    int64_t nacc = 0;
    for (int q = r0 * c->p.nx; q < r1 * c->p.nx; ++q) {
        if (cell_color(c, q) != color) {
            if (acc) acc[q] = -1;
            if (dec) dec[q] = 0.0;
            if (band) band[q] = 0.0;
            continue;
        }
        int a = trial(c, m, H, q, sweep, chain, seed, cos_tc, dec ? dec + q : NULL, band ? band + q : NULL);
        if (acc) acc[q] = (int8_t)a;
        nacc += a;
    }
    return nacc;
}

int64_t orc_pass(orc_ctx *c, double *m, const double *H, int color, uint32_t sweep,
                 uint32_t chain, uint64_t seed, double theta_deg,
                 int8_t *acc, double *dec, double *band)
{
    if (acc) for (int q = 0; q < c->n; ++q) acc[q] = -1;
    if (dec) for (int q = 0; q < c->n; ++q) dec[q] = 0.0;
    if (band) for (int q = 0; q < c->n; ++q) band[q] = 0.0;
    return pass_rows(c, m, H, color, 0, c->p.ny * c->p.nz, sweep, chain, seed, theta_deg, acc, dec, band);
}

/* App. B (Fig. 11): the size of each free-energy term of the trial moves.  For
 * every cell of the mesh (both sublattices, each against the same state m and
 * frozen field H) the trial move the sweep would propose at iteration `sweep`
 * (same random numbers, cone half-angle theta_deg) is drawn, its energy change
 * split into the terms of orc_local_dF, and |term| / kT of the cell averaged
 * over the cells: out = [ex, dmi, an, zee, long, demag]. */
void orc_trial_terms(orc_ctx *c, const double *m, const double *H, uint32_t sweep, uint32_t chain,
                     uint64_t seed, double theta_deg, double out[6])
{
    double cos_tc = cos(theta_deg * PI / 180.0);
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    for (int q = 0; q < c->n; ++q) {
        double u[4], mn[3], t[7];
        draw4((uint32_t)q + c->p.cell_base, sweep, chain, 0u, seed, u);
        propose(m + 3 * q, cos_tc, c->sigma[q], u, mn);
        orc_local_dF(c, m, H, q, mn, t);
        for (int k = 0; k < 6; ++k) out[k] += fabs(t[k + 1]) / c->kT[q];
    }
    for (int k = 0; k < 6; ++k) out[k] /= (double)c->n;
}

/* App. B: serial MMC, cells in index order, the demag field updated after
 * every accepted move so that every move's Eq. 14 term uses the field of the
 * current state (plus the self term when demag_self is set). */
int64_t orc_serial_sweep(orc_ctx *c, double *m, double *H, uint32_t sweep, uint32_t chain,
                         uint64_t seed, double theta_deg)
{
    double cos_tc = cos(theta_deg * PI / 180.0);
    const orc_problem *p = &c->p;
    int64_t nacc = 0;
    for (int q = 0; q < c->n; ++q) {
        double old[3] = {m[3 * q], m[3 * q + 1], m[3 * q + 2]};
        int a = trial(c, m, H, q, sweep, chain, seed, cos_tc, NULL, NULL);
        nacc += a;
        if (a && p->demag) {
            double dM[3] = {c->Ms0[q] * (m[3 * q] - old[0]), c->Ms0[q] * (m[3 * q + 1] - old[1]),
                            c->Ms0[q] * (m[3 * q + 2] - old[2])};
            int qi = q % p->nx, qj = (q / p->nx) % p->ny, qk = q / (p->nx * p->ny);
            for (int r = 0; r < c->n; ++r) {
                int ri = r % p->nx, rj = (r / p->nx) % p->ny, rk = r / (p->nx * p->ny);
                const double *t = c->Nt + 6 * toff(c, ri - qi, rj - qj, rk - qk);
                H[3 * r] -= t[0] * dM[0] + t[3] * dM[1] + t[4] * dM[2];
                H[3 * r + 1] -= t[3] * dM[0] + t[1] * dM[1] + t[5] * dM[2];
                H[3 * r + 2] -= t[4] * dM[0] + t[5] * dM[1] + t[2] * dM[2];
            }
        }
    }
    return nacc;
}

/* Sec. II: every 100 iterations, acceptance above 0.55 widens the cone by 1 deg,
 * below 0.45 narrows it by 1 deg; the half-angle stays in [1, 180] deg. */
double orc_adapt_theta(double theta_deg, int64_t acc, int64_t att)
{
    if (att <= 0) return theta_deg;
    double rate = (double)acc / (double)att;
    if (rate > 0.55) theta_deg += 1.0;
    else if (rate < 0.45) theta_deg -= 1.0;
    if (theta_deg < 1.0) theta_deg = 1.0;
    if (theta_deg > 180.0) theta_deg = 180.0;
    return theta_deg;
}

void orc_obs_accumulate(const orc_ctx *c, const double *m, orc_obs *obs)
{
    for (int q = 0; q < c->n; ++q) {
        const double *v = m + 3 * q;
        double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        obs->sum_m[0] += v[0]; obs->sum_m[1] += v[1]; obs->sum_m[2] += v[2];
        obs->sum_len += len;
        obs->sum_len2 += len * len;
        if (obs->hist && obs->hist_bins > 0) {
            int b = (int)(len / obs->hist_max * obs->hist_bins);
            if (b >= obs->hist_bins || b < 0) b = obs->hist_bins;
            obs->hist[b] += 1;
        }
    }
    obs->nsamples += c->n;
    obs->nsnap += 1;
}

/* Sec. II (Figs. 1-2): histogram of the vector lengths |m| of a state, in bins
 * equal bins on [0, hmax), lengths at or beyond hmax counted in hist[bins].
 * FP64: |m| = sqrt(x^2 + y^2 + z^2), bin = floor(|m| bins / hmax). */
void orc_hist(const double *m, int64_t n, int bins, double hmax, int64_t *hist)
{
    for (int b = 0; b <= bins; ++b) hist[b] = 0;
    for (int64_t q = 0; q < n; ++q) {
        const double *v = m + 3 * q;
        double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double t = len / hmax * bins;
        int b = t >= (double)bins ? bins : (int)t;
        hist[b] += 1;
    }
}

int64_t orc_run(orc_ctx *c, double *m, int64_t n, orc_run_state *st, orc_obs *obs, int obs_every)
{
    int64_t total = 0;
    double *H = NULL;
    if (c->p.demag && st->demag_mode > 0) H = (double *)calloc(3 * (size_t)c->n, sizeof(double));
    int method = c->n <= 1024 ? 0 : 1;
    for (int64_t s = 0; s < n; ++s) {
        int64_t acc = 0;
        if (st->demag_mode == 3) {
            /* App. B serial form: cells in index order; without demag it is the
               serial Metropolis sweep */
            if (H) orc_demag_field(c, m, H, method);
            acc = orc_serial_sweep(c, m, H, st->sweep, st->chain, st->seed, st->theta_deg);
        } else if (st->demag_mode == 2 && st->stripes > 1) {
            /* finer than per pass: each pass in `stripes` bands of rows, the
               demag field recomputed before every band */
            int nrows = c->p.ny * c->p.nz;
            for (int color = 0; color < 2; ++color)
                for (int k = 0; k < st->stripes; ++k) {
                    int r0 = (int)((int64_t)k * nrows / st->stripes);
                    int r1 = (int)((int64_t)(k + 1) * nrows / st->stripes);
                    if (H) orc_demag_field(c, m, H, method);
                    acc += pass_rows(c, m, H, color, r0, r1, st->sweep, st->chain, st->seed, st->theta_deg,
                                     NULL, NULL, NULL);
                }
        } else {
            if (H) orc_demag_field(c, m, H, method);
            acc += orc_pass(c, m, H, 0, st->sweep, st->chain, st->seed, st->theta_deg, NULL, NULL, NULL);
            if (H && st->demag_mode == 2) orc_demag_field(c, m, H, method);
            acc += orc_pass(c, m, H, 1, st->sweep, st->chain, st->seed, st->theta_deg, NULL, NULL, NULL);
        }
        total += acc;
        st->win_acc += acc;
        st->win_att += c->n;
        st->sweep += 1;
        if (st->sweep % 100 == 0) {
            if (st->adapt) st->theta_deg = orc_adapt_theta(st->theta_deg, st->win_acc, st->win_att);
            st->win_acc = 0; st->win_att = 0;
        }
        if (obs && obs_every > 0 && (s + 1) % obs_every == 0) orc_obs_accumulate(c, m, obs);
    }
    free(H);
    return total;
}

/* Initial state; the random form draws z = 2 u0 - 1, phi = 2 pi u1 from Philox
 * counter (cell, 0, chain, 1). */
void orc_init_state(const orc_ctx *c, double *m, int random, const double dir[3], double len,
                    uint32_t chain, uint64_t seed)
{
    double dl = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int q = 0; q < c->n; ++q) {
        if (random) {
            double u[4];
            draw4((uint32_t)q, 0u, chain, 1u, seed, u);
            double z = 2.0 * u[0] - 1.0, phi = 2.0 * PI * u[1];
            double r = sqrt(1.0 - z * z);
            m[3 * q] = len * r * cos(phi); m[3 * q + 1] = len * r * sin(phi); m[3 * q + 2] = len * z;
        } else {
            for (int a = 0; a < 3; ++a) m[3 * q + a] = len * dir[a] / dl;
        }
    }
}

/* ========================================================================== */
/* Gradient of the total energy (forward: orc_energy).                         */
void orc_energy_grad(orc_ctx *c, const double *m, double *g, double dEdp[5], double E[7])
{
    const orc_problem *p = &c->p;
    int n = c->n;
    memset(g, 0, sizeof(double) * 3 * (size_t)n);
    orc_energy(c, m, E);
    for (int k = 0; k < p->nz; ++k) for (int j = 0; j < p->ny; ++j) for (int i = 0; i < p->nx; ++i) {
        int q = i + p->nx * (j + p->ny * k);
        const double *mq = m + 3 * q;
        for (int a = 0; a < 3; ++a) {
            int r = neighbour(c, i, j, k, a, +1);
            if (r < 0) continue;
            double s = bond_scale(c, q, r);
            const double *mr = m + 3 * r;
            double cex = s * c->V * p->A0 / (p->h[a] * p->h[a]);
            for (int b = 0; b < 3; ++b) {
                g[3 * q + b] += 2.0 * cex * (mq[b] - mr[b]);
                g[3 * r + b] -= 2.0 * cex * (mq[b] - mr[b]);
            }
            if (a < 2) {
                double cd = s * c->V * p->D0 / p->h[a];
                /* E = -cd (mq_z mr_a - mq_a mr_z) with a the bond axis */
                g[3 * q + 2] += -cd * mr[a];
                g[3 * q + a] += cd * mr[2];
                g[3 * r + a] += -cd * mq[2];
                g[3 * r + 2] += cd * mq[a];
            }
        }
        double len = sqrt(mq[0] * mq[0] + mq[1] * mq[1] + mq[2] * mq[2]);
        if (len > 0.0) {
            double u[3] = {mq[0] / len, mq[1] / len, mq[2] / len};
            if (p->aniso_cubic) {
                /* d/du of V(K1 (a2b2 + a2g2 + b2g2) + K2 a2b2g2), projected */
                double a2 = u[0] * u[0], b2 = u[1] * u[1], g2 = u[2] * u[2];
                double du[3] = {
                    c->V * (c->K1T[q] * 2.0 * u[0] * (b2 + g2) + c->K2T[q] * 2.0 * u[0] * b2 * g2),
                    c->V * (c->K1T[q] * 2.0 * u[1] * (a2 + g2) + c->K2T[q] * 2.0 * u[1] * a2 * g2),
                    c->V * (c->K1T[q] * 2.0 * u[2] * (a2 + b2) + c->K2T[q] * 2.0 * u[2] * a2 * b2)};
                double dot = du[0] * u[0] + du[1] * u[1] + du[2] * u[2];
                for (int b = 0; b < 3; ++b) g[3 * q + b] += (du[b] - dot * u[b]) / len;
            } else {
                const double *e = c->eA + 3 * q;
                double d = u[0] * e[0] + u[1] * e[1] + u[2] * e[2];
                double coef = -2.0 * c->V * (c->K1T[q] + 2.0 * c->K2T[q] * (1.0 - d * d)) * d / len;
                for (int b = 0; b < 3; ++b) g[3 * q + b] += coef * (e[b] - d * u[b]);
            }
        }
        for (int b = 0; b < 3; ++b) g[3 * q + b] += -c->V * c->Ms0[q] * p->B[b];
        /* longitudinal (Eq. 7 exponent) */
        double T = c->T[q], Tc = c->Tc[q];
        double Tg = fabs(T - Tc) < 1e-3 ? (T < Tc ? Tc - 1e-3 : Tc + 1e-3) : T;
        double chi = c->chi[q];
        double coef;
        if (Tg < Tc) {
            double me2 = c->me[q] * c->me[q];
            coef = c->V * c->Ms0[q] * (len * len - me2) / (2.0 * chi * me2);
        } else {
            double cc = 3.0 * Tc / (10.0 * (Tg - Tc));
            coef = c->V * c->Ms0[q] / chi * (1.0 + 2.0 * cc * len * len);
        }
        for (int b = 0; b < 3; ++b) g[3 * q + b] += coef * mq[b];
    }
    if (p->demag) {
        double *H = (double *)malloc(sizeof(double) * 3 * (size_t)n);
        orc_demag_field(c, m, H, n <= 4096 ? 0 : 1);
        for (int q = 0; q < n; ++q)
            for (int b = 0; b < 3; ++b) g[3 * q + b] += -ORC_MU0 * c->V * c->Ms0[q] * H[3 * q + b];
        free(H);
    }
    /* parameter gradients (uniform material): E_ex ~ A0, E_dmi ~ D0, E_an ~ Ku,
     * E_l ~ 1/chi, E_l and E_Z ~ Ms0, E_d ~ Ms0^2 */
    double Ms = c->Ms0[0];
    dEdp[0] = (E[5] + E[4] + 2.0 * E[6]) / Ms;
    dEdp[1] = p->A0 != 0.0 ? E[1] / p->A0 : 0.0;
    dEdp[2] = p->D0 != 0.0 ? E[2] / p->D0 : 0.0;
    dEdp[3] = c->K1[0] != 0.0 ? E[3] / c->K1[0] : 0.0;
    dEdp[4] = c->chi[0] != 0.0 ? -E[5] / c->chi[0] : 0.0;
}


/* Sec. III comparison method (SDesc): zero-temperature steepest descent with
 * the lengths held at m_e(T) of each cell (the temperature enters only through
 * the rescaled parameters, as in the MMC energy).  With u_i = m_i / m_e,i unit
 * vectors, the tangential gradient is g_i = m_e,i (G_i - (G_i . u_i) u_i),
 * G = dE/dm; a step is u_i <- (u_i - tau g_i) / |u_i - tau g_i|.  tau: the first
 * step turns the cell with the largest gradient by 0.01 rad; afterwards the
 * Barzilai-Borwein step sizes s.s / s.y (odd steps) and s.y / y.y (even
 * steps) with s = u - u_prev, y = g - g_prev, keeping the previous tau when
 * s.y <= 0.  Stops when the largest normalized torque |u_i x h_i| / |h_i|
 * (h = -m_e G) is below tol. */
int orc_sdesc(orc_ctx *c, double *m, int maxit, double tol, int *iters, double *torque)
{
    const int n = c->n;
    double *u = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *up = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *G = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *g = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *gp = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *mm = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double dEdp[5], E[7];
    for (int q = 0; q < n; ++q) {
        double l = sqrt(m[3 * q] * m[3 * q] + m[3 * q + 1] * m[3 * q + 1] + m[3 * q + 2] * m[3 * q + 2]);
        for (int a = 0; a < 3; ++a) u[3 * q + a] = l > 0 ? m[3 * q + a] / l : (a == 0 ? 1.0 : 0.0);
    }
    double tau = 0.0, tmax = 0.0;
    int it = 0, done = 0;
    for (;;) {
        for (int q = 0; q < n; ++q)
            for (int a = 0; a < 3; ++a) mm[3 * q + a] = c->me[q] * u[3 * q + a];
        orc_energy_grad(c, mm, G, dEdp, E);
        double ss = 0, sy = 0, yy = 0, gmax = 0;
        tmax = 0.0;
        for (int q = 0; q < n; ++q) {
            const double *uq = u + 3 * q, *Gq = G + 3 * q;
            double me = c->me[q];
            double d = Gq[0] * uq[0] + Gq[1] * uq[1] + Gq[2] * uq[2];
            double gn2 = 0, Gn2 = 0;
            for (int a = 0; a < 3; ++a) {
                double ga = me * (Gq[a] - d * uq[a]);
                g[3 * q + a] = ga;
                gn2 += ga * ga;
                Gn2 += me * me * Gq[a] * Gq[a];
                double sa = uq[a] - up[3 * q + a], ya = ga - gp[3 * q + a];
                ss += sa * sa; sy += sa * ya; yy += ya * ya;
            }
            double r = Gn2 > 0 ? sqrt(gn2 / Gn2) : 0.0;   /* |u x h| / |h| */
            if (r > tmax) tmax = r;
            if (gn2 > gmax) gmax = gn2;
        }
        if (tmax < tol) { done = 1; break; }
        if (it >= maxit) break;
        if (it == 0) {
            tau = gmax > 0 ? 0.01 / sqrt(gmax) : 0.0;
        } else if (sy > 0) {
            tau = (it & 1) ? ss / sy : sy / yy;
        }
        for (int q = 0; q < n; ++q) {
            double v[3], l2 = 0;
            for (int a = 0; a < 3; ++a) {
                up[3 * q + a] = u[3 * q + a];
                gp[3 * q + a] = g[3 * q + a];
                v[a] = u[3 * q + a] - tau * g[3 * q + a];
                l2 += v[a] * v[a];
            }
            double il = 1.0 / sqrt(l2);
            for (int a = 0; a < 3; ++a) u[3 * q + a] = v[a] * il;
        }
        ++it;
    }
    for (int q = 0; q < n; ++q)
        for (int a = 0; a < 3; ++a) m[3 * q + a] = c->me[q] * u[3 * q + a];
    if (iters) *iters = it;
    if (torque) *torque = tmax;
    free(u); free(up); free(G); free(g); free(gp); free(mm);
    return done ? 0 : 1;
}


/* Sec. II, transverse distribution check (Fig. 1d-f): the polar angle of every
 * cell to the configuration's mean direction, histogrammed in bins equal
 * bins on [lo, hi); angles outside go to the last entry hist[bins].  FP64. */
void orc_angle_hist(const orc_ctx *c, const double *m, int bins, double lo, double hi, int64_t *hist,
                    double mean_dir[3])
{
    double s[3] = {0, 0, 0};
    for (int q = 0; q < c->n; ++q)
        for (int a = 0; a < 3; ++a) s[a] += m[3 * q + a];
    double l = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    double n[3] = {0, 0, 1};
    if (l > 0) for (int a = 0; a < 3; ++a) n[a] = s[a] / l;
    if (mean_dir) for (int a = 0; a < 3; ++a) mean_dir[a] = n[a];
    for (int b = 0; b <= bins; ++b) hist[b] = 0;
    for (int q = 0; q < c->n; ++q) {
        const double *v = m + 3 * q;
        double lv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double ct = lv > 0 ? (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / lv : 1.0;
        if (ct > 1.0) ct = 1.0;
        if (ct < -1.0) ct = -1.0;
        double th = acos(ct);
        double f = (th - lo) / (hi - lo) * bins;
        int b = (f >= 0.0 && f < (double)bins) ? (int)f : bins;
        hist[b] += 1;
    }
}
