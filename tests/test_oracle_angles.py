"""Oracle pins of the angular-deviation histogram (Sec. II, Fig. 1d-f: the
polar angle of every cell to the configuration's mean direction), CPU only.

- A uniform state: every angle is 0 (first bin).
- Directions uniform on a cap of half-angle alpha about z: the mean points
  along z and the angle density is sin(theta) / (1 - cos alpha) on [0, alpha]
  (chi-square against the bin integrals).
- Directions uniform on the sphere (mean of a large sample nearly 0): the
  density about any axis is sin(theta) / 2.
- Lengths do not matter (directions only); angles outside [lo, hi) go to the
  overflow entry.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _cap_sample(n, alpha, rng):
    ct = 1.0 - rng.uniform(0, 1, n) * (1.0 - math.cos(alpha))
    ph = rng.uniform(0, 2 * math.pi, n)
    st = np.sqrt(1 - ct * ct)
    return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)


def _chi2_p(obs, expected):
    from scipy.stats import chi2
    sel = expected > 5
    x = ((obs[sel] - expected[sel]) ** 2 / expected[sel]).sum()
    return chi2.sf(x, sel.sum() - 1)


def test_uniform_state_is_all_zero_angle():
    s = W._base((8, 8, 1), (4e-9,) * 3)
    h, d = O.Oracle(s).angle_hist(np.tile([0.3, 0.4, 0.0], (64, 1)) * 2.0, bins=10)
    assert h[0] == 64 and h[1:].sum() == 0
    assert np.allclose(d, [0.6, 0.8, 0.0])


@pytest.mark.parametrize("alpha_deg", [20.0, 90.0])
def test_cap_distribution(alpha_deg):
    alpha = math.radians(alpha_deg)
    n = 128 * 128
    rng = np.random.default_rng(7)
    u = _cap_sample(n, alpha, rng) * rng.uniform(0.5, 1.0, (n, 1))
    s = W._base((128, 128, 1), (4e-9,) * 3)
    bins = 50
    h, d = O.Oracle(s).angle_hist(u, bins=bins, lo=0.0, hi=alpha)
    assert d[2] > 0.99
    edges = np.linspace(0.0, alpha, bins + 1)
    expected = n * (np.cos(edges[:-1]) - np.cos(edges[1:])) / (1 - math.cos(alpha))
    assert h[bins] <= 0.01 * n           # the sample mean is tilted from z: a few angles exceed alpha
    assert _chi2_p(h[:bins], expected) > 1e-3


def test_isotropic_distribution_and_overflow():
    n = 160 * 160
    rng = np.random.default_rng(3)
    v = rng.standard_normal((n, 3))
    s = W._base((160, 160, 1), (4e-9,) * 3)
    bins = 40
    h, _ = O.Oracle(s).angle_hist(v, bins=bins, lo=0.0, hi=math.pi)
    edges = np.linspace(0.0, math.pi, bins + 1)
    expected = n * (np.cos(edges[:-1]) - np.cos(edges[1:])) / 2
    assert h[bins] == 0
    assert _chi2_p(h[:bins], expected) > 1e-3
    h2, _ = O.Oracle(s).angle_hist(v, bins=bins, lo=0.0, hi=math.pi / 2)
    assert h2[:bins].sum() + h2[bins] == n and h2[bins] > 0.4 * n
