"""Pins of the oracle's deterministic parts against what the paper and the
mathematics fix (CPU only).

- Philox4x32-10: published known-answer vectors.
- Eqs. 8-9: asymptotes and closed forms of m_e(T) and chi(T).
- Eq. 13: sigma is one standard deviation of the Gaussian in m^2 of Eq. 7.
- Eq. 11 / Eq. 12 values at special directions, the m_e^{l(l+1)/2} law.
- Sec. II cone adaptation rule.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

KB = O.KB
MUB = O.MUB
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert O.philox(r[0:4], r[4:6]) == r[6:10]


def test_uniform_range_and_exactness():
    lo, hi = O.u01(0), O.u01(0xFFFFFFFF)
    assert lo == 0.5 * 2.0 ** -23 and hi == 1.0 - 0.5 * 2.0 ** -23
    for r in (0, 511, 512, 12345678, 0xDEADBEEF, 0xFFFFFFFF):
        u = O.u01(r)
        assert np.float64(np.float32(u)) == u          # exact in FP32
        assert u == ((r >> 9) + 0.5) / 8388608.0


@pytest.mark.parametrize("T,Tc", [(1.0, 870.0), (10.0, 870.0), (5.0, 600.0)])
def test_me_low_temperature_closed_form(T, Tc):
    # for large x, B(x) = 1 - 1/x up to exp(-2x): m = 1 - T/(3 Tc m)
    t = T / (3.0 * Tc)
    assert O.me(T, Tc) == pytest.approx((1.0 + math.sqrt(1.0 - 4.0 * t)) / 2.0, abs=2e-15)


@pytest.mark.parametrize("T,Tc", [(300, 870), (800, 870), (50, 600), (570, 600), (869.0, 870)])
def test_me_fixed_point_residual(T, Tc):
    m = O.me(T, Tc)
    assert 0.0 < m < 1.0
    assert abs(O.langevin(3.0 * Tc * m / T) - m) < 1e-15


@pytest.mark.parametrize("eps", [1e-4, 1e-5])
def test_me_near_tc(eps):
    # Taylor of B: m_e^2 -> (5/3)(1 - T/Tc) as T -> Tc-
    Tc = 870.0
    T = Tc * (1.0 - eps)
    ratio = O.me(T, Tc) ** 2 / (5.0 / 3.0 * eps)
    assert abs(ratio - 1.0) < 5 * eps


def test_me_above_tc_is_zero():
    assert O.me(900.0, 870.0) == 0.0
    assert O.me(870.0, 870.0) == 0.0    # evaluated 1 mK above (guard), on the T >= Tc side


@pytest.mark.parametrize("T", [871.0, 900.0, 1200.0])
def test_chi_above_tc_closed_form(T):
    Tc = 870.0
    assert O.chi(T, Tc) == pytest.approx(MUB / (3.0 * KB * (T - Tc)), rel=1e-13)


@pytest.mark.parametrize("eps", [1e-4, 1e-5])
def test_chi_below_tc_asymptote(eps):
    Tc = 870.0
    T = Tc * (1.0 - eps)
    ratio = O.chi(T, Tc) / (MUB / (6.0 * KB * (Tc - T)))
    assert abs(ratio - 1.0) < 10 * eps


def test_chi_positive_and_decreasing_far_below_tc():
    vals = [O.chi(T, 870.0) for T in (100, 200, 300, 500, 700)]
    assert all(v > 0 for v in vals)
    assert all(a < b for a, b in zip(vals, vals[1:]))   # grows toward Tc


@pytest.mark.parametrize("T,Tc,h,Ms0", [(300, 870, 5e-9, 8.6e5), (300, 870, 4e-9, 8.6e5),
                                        (50, 600, 2e-9, 6e5), (800, 870, 5e-9, 8.6e5)])
def test_sigma_is_gaussian_width_of_eq7(T, Tc, h, Ms0):
    # Eq. 13 sigma is the standard deviation of the Gaussian in m^2 of Eq. 7:
    # the Eq. 7 exponent is exactly 1/2 at m^2 = m_e^2 + sigma (uncapped case)
    V = h ** 3 if h != 2e-9 else 2e-9 * 2e-9 * 1e-9
    s = O.sigma(T, Tc, V, Ms0, cap=1.0)
    m = math.sqrt(O.me(T, Tc) ** 2 + s)
    assert O.long_energy(m, T, Tc, V, Ms0) / (KB * T) == pytest.approx(0.5, rel=1e-12)
    assert O.sigma(T, Tc, V, Ms0) == min(s, 0.03)


def test_sigma_capped_at_and_above_tc():
    assert O.sigma(900, 870, 1e-25, 8.6e5) == 0.03
    assert O.sigma(600, 600, 4e-27, 6e5) == 0.03
    assert O.sigma(590, 600, 4e-27, 6e5) == 0.03      # close to Tc the cap is reached


def test_long_energy_above_tc_form():
    # T > Tc branch: quadratic + quartic in m with chi = mu/(3 kB (T - Tc))
    T, Tc, V, Ms0 = 650.0, 600.0, 4e-27, 6e5
    chi = MUB / (3 * KB * (T - Tc))
    for m in (0.01, 0.1, 0.3):
        ref = V * Ms0 * m * m / (2 * chi) * (1 + 3 * Tc * m * m / (10 * (T - Tc)))
        assert O.long_energy(m, T, Tc, V, Ms0) == pytest.approx(ref, rel=1e-13)
    # below Tc the minimum is at m_e with value 0
    me = O.me(300, 870)
    assert O.long_energy(me, 300, 870, 1e-25, 8.6e5) == 0.0


def _single(spec_over):
    import workloads as W
    s = W._base((2, 1, 1), (5e-9, 5e-9, 5e-9), A0=0.0)
    s.update(spec_over)
    return O.Oracle(s)


def test_anisotropy_special_directions():
    Ku, K2 = 4e5, 1e5
    o = _single({"K1": Ku, "K2": K2, "eA": (0.0, 0.0, 1.0)})
    tb = o.tables()
    me = O.me(300, 870)
    assert tb["K1T"][0] == pytest.approx(Ku * me ** 3, rel=1e-14)      # l = 2
    assert tb["K2T"][0] == pytest.approx(K2 * me ** 10, rel=1e-14)     # l = 4
    V = 125e-27
    par = np.array([[0, 0, 0.7], [0, 0, -0.7]])
    perp = np.array([[0.7, 0, 0], [0, 0.5, 0]])
    assert o.energy(par)[3] == pytest.approx(0.0, abs=1e-40)
    assert o.energy(perp)[3] == pytest.approx(2 * V * (tb["K1T"][0] + tb["K2T"][0]), rel=1e-13)


def test_cubic_anisotropy_special_directions():
    K1, K2 = 4.8e4, -1e4
    o = _single({"K1": K1, "K2": K2, "aniso": "cubic"})
    tb = o.tables()
    me = O.me(300, 870)
    assert tb["K1T"][0] == pytest.approx(K1 * me ** 10, rel=1e-13)     # l = 4
    assert tb["K2T"][0] == pytest.approx(K2 * me ** 21, rel=1e-13)     # l = 6
    V = 125e-27
    s = 0.8 / math.sqrt(3)
    diag = np.array([[s, s, s], [1.0, 0, 0]])
    E = o.energy(diag)[3]
    assert E == pytest.approx(V * (tb["K1T"][0] / 3 + tb["K2T"][0] / 27), rel=1e-12)


def test_zeeman_value():
    o = _single({"B": (0.01, 0.0, 0.0), "Ms0": 8.6e5})
    m = np.array([[0.8, 0, 0], [0, 0.8, 0]])
    assert o.energy(m)[4] == pytest.approx(-125e-27 * 8.6e5 * 0.8 * 0.01, rel=1e-14)


@pytest.mark.parametrize("theta,acc,att,exp", [
    (30.0, 56, 100, 31.0), (30.0, 44, 100, 29.0), (30.0, 50, 100, 30.0),
    (30.0, 55, 100, 30.0), (30.0, 45, 100, 30.0), (1.0, 0, 100, 1.0), (180.0, 100, 100, 180.0)])
def test_cone_adaptation_rule(theta, acc, att, exp):
    assert O.adapt_theta(theta, acc, att) == exp


def test_hist_counts_of_known_lengths():
    """The |m| histogram (Sec. II, Figs. 1-2) of states whose lengths are known
    exactly: c_b cells at the centre of bin b land in bin b, lengths at or above
    hmax in the overflow entry, for any direction; doubling hmax halves the bin
    index."""
    rng = np.random.default_rng(3)
    bins, hmax = 200, 1.0
    counts = rng.integers(0, 7, bins)
    L = np.repeat((np.arange(bins) + 0.5) * hmax / bins, counts)
    L = np.concatenate([L, [1.0, 1.0 + 1e-9, 1.3]])          # overflow: at and beyond hmax
    d = rng.standard_normal((L.size, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    m = d * L[:, None]
    h = O.hist(m, bins, hmax)
    assert np.array_equal(h[:bins], counts)
    assert h[bins] == 3
    # a zero vector is in bin 0; hmax = 2 maps centre (b + 1/2)/200 to bin b // 2
    # (t = b/2 + 1/4), and the lengths 1, 1 + 1e-9, 1.3 to bins 100, 100, 130
    assert O.hist(np.zeros((4, 3)), bins, hmax)[0] == 4
    h2 = O.hist(m, bins, 2.0)
    exp = np.zeros(bins + 1, np.int64)
    for b in range(bins):
        exp[b // 2] += counts[b]
    exp[100] += 2
    exp[130] += 1
    assert np.array_equal(h2, exp)
