// Host-side FP64 physics of the MMC method: thermodynamic tables (Sec. II,
// Eqs. 7-9, 13) and the demagnetizing-tensor spectra (Sec. III, Eq. 14).
// Runs once per create / temperature change; nothing here is on the sweep path.
#include <algorithm>
#include <cmath>
#include <complex>
#include <thread>
#include <vector>

#include "mmc_internal.h"

namespace mmc {

// ---------------------------------------------------------------------------
// Langevin function B(x) = coth x - 1/x and its derivative (Eq. 8).  Below
// |x| = 2 B is evaluated from Lambert's continued fraction of coth,
// coth x - 1/x = x / (3 + x^2 / (5 + x^2 / (7 + ...))), which has no
// cancellation; B' = 1 - B^2 - 2 B / x follows from d coth / dx = 1 - coth^2.
double langevin(double x) {
  if (std::fabs(x) < 2.0) {
    const double x2 = x * x;
    double d = 2.0 * 24 + 3.0;
    for (int k = 24; k >= 1; --k) d = (2.0 * k + 1.0) + x2 / d;
    return x / d;
  }
  return std::cosh(x) / std::sinh(x) - 1.0 / x;
}

double langevin_deriv(double x) {
  const double a = std::fabs(x);
  if (a == 0.0) return 1.0 / 3.0;
  if (a < 2.0) {
    const double L = langevin(x);
    return 1.0 - L * L - 2.0 * L / x;
  }
  if (a > 30.0) return 1.0 / (x * x);
  const double s = std::sinh(x);
  return 1.0 / (x * x) - 1.0 / (s * s);
}

static double guard_T(double T, double Tc) {
  if (std::fabs(T - Tc) < 1e-3) return T < Tc ? Tc - 1e-3 : Tc + 1e-3;
  return T;
}

// Eq. 9 at zero field: the positive root of g(m) = B(b m) - m, b = 3 Tc / T.
// g is concave on m > 0, so Newton from m = 1 descends monotonically onto it.
double me_of_T(double T, double Tc) {
  T = guard_T(T, Tc);
  if (T >= Tc) return 0.0;
  const double b = 3.0 * Tc / T;
  double m = 1.0;
  for (int it = 0; it < 500; ++it) {
    const double g = langevin(b * m) - m;
    const double gp = b * langevin_deriv(b * m) - 1.0;
    const double next = m - g / gp;
    if (!(next > 0.0) || !(next <= 1.0)) break;
    if (std::fabs(next - m) <= 1e-17 * m) { m = next; return m; }
    m = next;
  }
  // fallback: bisection on (0, 1]
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 1100 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (langevin(b * mid) > mid) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// Eq. 8 (1/T).
double chi_of_T(double T, double Tc, double mu) {
  T = guard_T(T, Tc);
  const double me = me_of_T(T, Tc);
  const double x = 3.0 * Tc * me / T;
  const double d = langevin_deriv(x);
  return mu / (kB * T) * d / (1.0 - 3.0 * Tc / T * d);
}

// Eq. 13, capped; the cap also applies at and above Tc.
double sigma_of_T(double T, double Tc, double mu, double V, double Ms0, double cap) {
  T = guard_T(T, Tc);
  if (T >= Tc) return cap;
  const double s = 2.0 * me_of_T(T, Tc) * std::sqrt(chi_of_T(T, Tc, mu) * kB * T / (V * Ms0));
  return std::min(s, cap);
}

// Eq. 7 exponent times kT as a polynomial in m^2 (constant dropped).
void long_coeffs(double T, double Tc, double mu, double V, double Ms0, double *c2, double *c4) {
  T = guard_T(T, Tc);
  const double chi = chi_of_T(T, Tc, mu);
  if (T < Tc) {
    const double me = me_of_T(T, Tc);
    const double a = V * Ms0 / (8.0 * chi * me * me);
    *c4 = a;
    *c2 = -2.0 * a * me * me;
  } else {
    *c2 = V * Ms0 / (2.0 * chi);
    *c4 = *c2 * 3.0 * Tc / (10.0 * (T - Tc));
  }
}

// sqrt(<m^2>) of the Eq. 7 length distribution (Simpson on a fine grid).
double rms_len_eq7(double T, double Tc, double mu, double V, double Ms0) {
  double c2, c4;
  long_coeffs(T, Tc, mu, V, Ms0, &c2, &c4);
  const double kT = kB * guard_T(T, Tc);
  const int n = 20000;
  const double mmax = 1.5;
  double s0 = 0.0, s2 = 0.0, fmin = 1e300;
  for (int i = 0; i <= n; ++i) {
    const double m = mmax * i / n, q = m * m;
    fmin = std::min(fmin, (c2 * q + c4 * q * q) / kT);
  }
  for (int i = 0; i <= n; ++i) {
    const double m = mmax * i / n, q = m * m;
    const double w = (i == 0 || i == n) ? 1.0 : (i % 2 ? 4.0 : 2.0);
    const double p = q * std::exp(-((c2 * q + c4 * q * q) / kT - fmin));
    s0 += w * p;
    s2 += w * p * q;
  }
  return std::sqrt(s2 / s0);
}

// ---------------------------------------------------------------------------
// Demagnetizing tensor.
//
// Near field: Newell, Williams & Dunlop's closed forms f (diagonal) and g
// (off-diagonal) combined over the 3x3x3 neighbourhood with weights
// (2, -1, -1) per axis.  Their cancellation grows like (R/h)^5.6 (about 1e-9
// relative at 11 cells in FP64), so beyond 6 h_max the cell-pair average of
// the point-dipole kernel is integrated
// numerically instead: the difference of two uniform points in two cells has a
// triangular density per axis, integrated by Gauss-Legendre on each half.

static double newell_f(double x, double y, double z) {
  x = std::fabs(x); y = std::fabs(y); z = std::fabs(z);
  const double xx = x * x, yy = y * y, zz = z * z;
  const double R = std::sqrt(xx + yy + zz);
  if (R == 0.0) return 0.0;
  double s = (2.0 * xx - yy - zz) * R / 6.0;
  const double rxz = std::sqrt(xx + zz), rxy = std::sqrt(xx + yy);
  if (y > 0.0 && rxz > 0.0) s += 0.5 * y * (zz - xx) * std::asinh(y / rxz);
  if (z > 0.0 && rxy > 0.0) s += 0.5 * z * (yy - xx) * std::asinh(z / rxy);
  if (x > 0.0 && y > 0.0 && z > 0.0) s -= x * y * z * std::atan(y * z / (x * R));
  return s;
}

static double newell_g(double x, double y, double z) {
  double sign = 1.0;
  if (x < 0.0) { sign = -sign; x = -x; }
  if (y < 0.0) { sign = -sign; y = -y; }
  z = std::fabs(z);
  if (x == 0.0 || y == 0.0) return 0.0;
  const double xx = x * x, yy = y * y, zz = z * z;
  const double R = std::sqrt(xx + yy + zz);
  double s = -x * y * R / 3.0;
  s += y * (3.0 * zz - yy) / 6.0 * std::asinh(x / std::sqrt(yy + zz));
  s += x * (3.0 * zz - xx) / 6.0 * std::asinh(y / std::sqrt(xx + zz));
  if (z > 0.0) {
    s += x * y * z * std::asinh(z / std::sqrt(xx + yy));
    s -= zz * z / 6.0 * std::atan(x * y / (z * R));
    s -= z * yy / 2.0 * std::atan(x * z / (y * R));
    s -= z * xx / 2.0 * std::atan(y * z / (x * R));
  }
  return sign * s;
}

template <typename F>
static double second_diff3(F fn, double X, double Y, double Z, double a, double b, double c) {
  double s = 0.0;
  for (int i = -1; i <= 1; ++i) {
    const double wi = i == 0 ? 2.0 : -1.0;
    for (int j = -1; j <= 1; ++j) {
      const double wj = j == 0 ? 2.0 : -1.0;
      for (int k = -1; k <= 1; ++k) {
        const double wk = k == 0 ? 2.0 : -1.0;
        s += wi * wj * wk * fn(X + i * a, Y + j * b, Z + k * c);
      }
    }
  }
  return s;
}

static void newell_tensor(const double h[3], const double R[3], double out[6]) {
  const double norm = 1.0 / (4.0 * kPi * h[0] * h[1] * h[2]);
  const double X = R[0], Y = R[1], Z = R[2];
  out[0] = norm * second_diff3(newell_f, X, Y, Z, h[0], h[1], h[2]);
  out[1] = norm * second_diff3(newell_f, Y, X, Z, h[1], h[0], h[2]);
  out[2] = norm * second_diff3(newell_f, Z, Y, X, h[2], h[1], h[0]);
  out[3] = norm * second_diff3(newell_g, X, Y, Z, h[0], h[1], h[2]);
  out[4] = norm * second_diff3(newell_g, X, Z, Y, h[0], h[2], h[1]);
  out[5] = norm * second_diff3(newell_g, Y, Z, X, h[1], h[2], h[0]);
}

struct TriRule {
  int n = 0;
  double u[24], w[24];
};

// Nodes on [-1, 1] of the n-point Gauss-Legendre rule (Newton on P_n).
static void gl_nodes(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double t = std::cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (p0 - t * p1) / (1.0 - t * t);
      const double step = p1 / dp;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// rule for E[f(u)], u with density (d - |u|)/d^2 on [-d, d]
static TriRule tri_rule(double d, int n) {
  TriRule r;
  double x[12], w[12];
  gl_nodes(n, x, w);
  for (int side = -1; side <= 1; side += 2)
    for (int i = 0; i < n; ++i) {
      const double t = 0.5 * d * (1.0 + x[i]);
      r.u[r.n] = side * t;
      r.w[r.n] = 0.5 * d * w[i] * (d - t) / (d * d);
      ++r.n;
    }
  return r;
}

static void dipole_average(const double h[3], const double R[3], const TriRule q[3], double out[6]) {
  double a[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < q[0].n; ++i)
    for (int j = 0; j < q[1].n; ++j) {
      const double wij = q[0].w[i] * q[1].w[j];
      const double rx = R[0] + q[0].u[i], ry = R[1] + q[1].u[j];
      for (int k = 0; k < q[2].n; ++k) {
        const double rz = R[2] + q[2].u[k];
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double inv = 1.0 / r2;
        const double w = wij * q[2].w[k] * inv * inv / std::sqrt(r2);
        a[0] += w * (3.0 * rx * rx - r2);
        a[1] += w * (3.0 * ry * ry - r2);
        a[2] += w * (3.0 * rz * rz - r2);
        a[3] += w * 3.0 * rx * ry;
        a[4] += w * 3.0 * rx * rz;
        a[5] += w * 3.0 * ry * rz;
      }
    }
  const double pref = -h[0] * h[1] * h[2] / (4.0 * kPi);
  for (int c = 0; c < 6; ++c) out[c] = pref * a[c];
}

struct TensorRules {
  TriRule r8[3], r6[3], r4[3], r3[3], r2[3];
  explicit TensorRules(const double h[3]) {
    for (int a = 0; a < 3; ++a) {
      r8[a] = tri_rule(h[a], 8);
      r6[a] = tri_rule(h[a], 6);
      r4[a] = tri_rule(h[a], 4);
      r3[a] = tri_rule(h[a], 3);
      r2[a] = tri_rule(h[a], 2);
    }
  }
};

// n Gauss points per half integrate the cell-pair average with a relative error
// of order (h/R)^(2n); the ladder keeps it below ~1e-12 (1e-10 from 300 h on,
// where only far offsets and periodic images fall)
static void tensor_with(const double h[3], const double R[3], const TensorRules &rules, double out[6]) {
  const double hmax = std::max(h[0], std::max(h[1], h[2]));
  const double r = std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]) / hmax;
  if (r < 6.0) newell_tensor(h, R, out);
  else if (r < 12.0) dipole_average(h, R, rules.r8, out);
  else if (r < 40.0) dipole_average(h, R, rules.r6, out);
  else if (r < 100.0) dipole_average(h, R, rules.r4, out);
  else if (r < 300.0) dipole_average(h, R, rules.r3, out);
  else dipole_average(h, R, rules.r2, out);
}

void demag_tensor(const double h[3], const double R[3], double out[6]) {
  TensorRules rules(h);
  tensor_with(h, R, rules, out);
}

// in-place radix-2 complex FFT (forward), stride s
static void fft_inplace(std::complex<double> *a, int n, long long s) {
  if (n <= 1) return;
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    while (j & bit) { j ^= bit; bit >>= 1; }
    j |= bit;
    if (i < j) std::swap(a[i * s], a[j * s]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1;
    for (int k = 0; k < half; ++k) {
      const double ang = -2.0 * kPi * k / len;
      const std::complex<double> w(std::cos(ang), std::sin(ang));
      for (int i = k; i < n; i += len) {
        const std::complex<double> u = a[i * s], v = w * a[(i + half) * s];
        a[i * s] = u + v;
        a[(i + half) * s] = u - v;
      }
    }
  }
}

template <typename F>
static void parallel_for(long long total, F fn) {
  const int nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back([&, t]() {
      for (long long q = t; q < total; q += nth) fn(q);
    });
  for (auto &x : th) x.join();
}

// Periodic kernel at base offsets 0 <= d_a <= n_a / 2 along the periodic axes
// (0 <= d_a < o_a along open ones): the tensor summed over the images
// d_a + p n_a, |p| <= images, the half period d_a = n_a / 2 split between
// +n_a / 2 and -n_a / 2 with weight 1/2 each.
static void periodic_base(const double h[3], const DemagPeriodic &pd, const TensorRules &rules, int bx, int by,
                          int bz, std::vector<double> &base) {
  parallel_for(1LL * bx * by * bz, [&](long long q) {
    const int d[3] = {(int)(q % bx), (int)((q / bx) % by), (int)(q / (1LL * bx * by))};
    int nrep[3], rep[3][2], P[3];
    double w[3][2];
    for (int a = 0; a < 3; ++a) {
      const bool per = pd.images > 0 && pd.per[a];
      P[a] = per ? pd.images : 0;
      rep[a][0] = d[a];
      w[a][0] = 1.0;
      nrep[a] = 1;
      if (per && 2 * d[a] == pd.n[a]) {
        nrep[a] = 2;
        rep[a][1] = -d[a];
        w[a][0] = w[a][1] = 0.5;
      }
    }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nrep[0]; ++i)
      for (int j = 0; j < nrep[1]; ++j)
        for (int k = 0; k < nrep[2]; ++k) {
          const double wt = w[0][i] * w[1][j] * w[2][k];
          for (int pz = -P[2]; pz <= P[2]; ++pz)
            for (int py = -P[1]; py <= P[1]; ++py)
              for (int px = -P[0]; px <= P[0]; ++px) {
                const double R[3] = {(rep[0][i] + px * pd.n[0]) * h[0], (rep[1][j] + py * pd.n[1]) * h[1],
                                     (rep[2][k] + pz * pd.n[2]) * h[2]};
                double t[6];
                tensor_with(h, R, rules, t);
                for (int c = 0; c < 6; ++c) acc[c] += wt * t[c];
              }
        }
    // at a half period the components odd in that axis cancel exactly (parity)
    static const int odd[3][6] = {{0, 0, 0, 1, 1, 0}, {0, 0, 0, 1, 0, 1}, {0, 0, 0, 0, 1, 1}};
    for (int a = 0; a < 3; ++a)
      if (nrep[a] == 2)
        for (int c = 0; c < 6; ++c)
          if (odd[a][c]) acc[c] = 0.0;
    for (int c = 0; c < 6; ++c) base[6 * q + c] = acc[c];
  });
}

// the six tensor components (xx yy zz xy xz yz) at offsets (x, y, z) h with
// 0 <= x < ox, 0 <= y < oy, 0 <= z < oz, interleaved: oct[6 (x + ox (y + oy z)) + c];
// the other octants follow by symmetry (xy odd in x and y, xz in x and z, yz in y and z).
// Along a periodic axis of pd the value at x is the periodic kernel at x mod n,
// taken from its base offset min(r, n - r), r = x mod n, with the sign of the
// components odd in that axis flipped when r > n / 2 (the kernel is periodic and
// has the tensor's parity).
void demag_octant(const double h[3], int ox, int oy, int oz, std::vector<double> &oct, const DemagPeriodic &pd) {
  oct.assign((size_t)6 * ox * oy * oz, 0.0);
  TensorRules rules(h);
  if (!pd.any()) {
    parallel_for(1LL * ox * oy * oz, [&](long long q) {
      const int x = (int)(q % ox), y = (int)((q / ox) % oy), z = (int)(q / (1LL * ox * oy));
      const double R[3] = {x * h[0], y * h[1], z * h[2]};
      tensor_with(h, R, rules, &oct[6 * q]);
    });
    return;
  }
  const int o[3] = {ox, oy, oz};
  bool per[3];
  int b[3];
  for (int a = 0; a < 3; ++a) {
    per[a] = pd.per[a] != 0;
    b[a] = per[a] ? pd.n[a] / 2 + 1 : o[a];
  }
  std::vector<double> base((size_t)6 * b[0] * b[1] * b[2]);
  periodic_base(h, pd, rules, b[0], b[1], b[2], base);
  // odd components per axis: xy (3) in x, y; xz (4) in x, z; yz (5) in y, z
  static const int odd[3][6] = {{0, 0, 0, 1, 1, 0}, {0, 0, 0, 1, 0, 1}, {0, 0, 0, 0, 1, 1}};
  for (int z = 0; z < oz; ++z)
    for (int y = 0; y < oy; ++y)
      for (int x = 0; x < ox; ++x) {
        const int v[3] = {x, y, z};
        int d[3];
        bool flip[3] = {false, false, false};
        for (int a = 0; a < 3; ++a) {
          d[a] = v[a];
          if (per[a]) {
            const int r = v[a] % pd.n[a];
            flip[a] = 2 * r > pd.n[a];
            d[a] = flip[a] ? pd.n[a] - r : r;
          }
        }
        const double *src = &base[6 * (d[0] + 1LL * b[0] * (d[1] + 1LL * b[1] * d[2]))];
        double *dst = &oct[6 * (x + 1LL * ox * (y + 1LL * oy * z))];
        for (int c = 0; c < 6; ++c) {
          double s = 1.0;
          for (int a = 0; a < 3; ++a)
            if (flip[a] && odd[a][c]) s = -s;
          dst[c] = s * src[c];
        }
      }
}

void demag_spectra(const double h[3], int Px, int Py, int Pz, std::vector<double> &out, const DemagPeriodic &pd) {
  const int ncomp = Pz > 1 ? 6 : 4;
  const int qx = Px / 2 + 1, qy = Py / 2 + 1, qz = Pz / 2 + 1;
  const long long P = 1LL * Px * Py * Pz;
  const long long Q = 1LL * qx * qy * qz;
  out.assign((size_t)ncomp * Q, 0.0);

  // tensor on the symmetric octant of offsets |X| < Px/2, ... (on a padded axis
  // the Nyquist offset -P/2 never reaches a mesh cell when n <= P/2 and is left
  // at zero, which keeps every spectrum real; on a circular axis, P = n, it is
  // the periodic kernel's half-period value, whose odd components vanish)
  const int ox = pd.circ[0] ? Px / 2 + 1 : std::max(Px / 2, 1);
  const int oy = pd.circ[1] ? Py / 2 + 1 : std::max(Py / 2, 1);
  const int oz = pd.circ[2] ? Pz / 2 + 1 : std::max(Pz / 2, 1);
  std::vector<double> oct;
  demag_octant(h, ox, oy, oz, oct, pd);
  static const int comp_map[6] = {0, 1, 2, 3, 4, 5};  // xx yy zz xy xz yz
  std::vector<std::complex<double>> a((size_t)P);
  for (int c = 0; c < ncomp; ++c) {
    const int cc = comp_map[c];
    for (int z = 0; z < Pz; ++z)
      for (int y = 0; y < Py; ++y)
        for (int x = 0; x < Px; ++x) {
          const int X = x < (Px + 1) / 2 ? x : x - Px;
          const int Y = y < (Py + 1) / 2 ? y : y - Py;
          const int Z = z < (Pz + 1) / 2 ? z : z - Pz;
          double v = 0.0;
          const bool nyq = (Px > 1 && !pd.circ[0] && X == -Px / 2) || (Py > 1 && !pd.circ[1] && Y == -Py / 2) ||
                           (Pz > 1 && !pd.circ[2] && Z == -Pz / 2);
          if (!nyq) {
            const int ax = std::abs(X), ay = std::abs(Y), az = std::abs(Z);
            v = oct[6 * (ax + 1LL * ox * (ay + 1LL * oy * az)) + cc];
            const int sx = X < 0 ? -1 : 1, sy = Y < 0 ? -1 : 1, sz = Z < 0 ? -1 : 1;
            if (cc == 3) v *= sx * sy;
            if (cc == 4) v *= sx * sz;
            if (cc == 5) v *= sy * sz;
          }
          a[x + 1LL * Px * (y + 1LL * Py * z)] = v;
        }
    for (int z = 0; z < Pz; ++z)
      for (int y = 0; y < Py; ++y) fft_inplace(&a[1LL * Px * (y + 1LL * Py * z)], Px, 1);
    for (int z = 0; z < Pz; ++z)
      for (int x = 0; x < Px; ++x) fft_inplace(&a[x + 1LL * Px * Py * z], Py, Px);
    for (int y = 0; y < Py; ++y)
      for (int x = 0; x < Px; ++x) fft_inplace(&a[x + 1LL * Px * y], Pz, 1LL * Px * Py);
    for (int z = 0; z < qz; ++z)
      for (int y = 0; y < qy; ++y)
        for (int x = 0; x < qx; ++x)
          out[(size_t)c * Q + x + 1LL * qx * (y + 1LL * qy * z)] =
              a[(x % Px) + 1LL * Px * ((y % Py) + 1LL * Py * (z % Pz))].real();
  }
}

}  // namespace mmc
