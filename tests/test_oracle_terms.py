"""Oracle pins for the per-term size of the trial moves (App. B, Fig. 11): the
mean |dF_term| / kT over the trial moves of every cell.

In a uniform state m = m0 x (all cells equal) the trial move of a cell changes
- the exchange pair energy by 4 c_ex |m' - m|^2 (2D, four equal neighbours),
  whose mean over the proposal is 4 c_ex m0^2 (sigma^2 / 3 + 1 - cos theta);
- the Zeeman energy (B along x) by V Ms0 B m0 (1 - s cos t), whose mean
  magnitude is V Ms0 B m0 (1 - cos theta) / 2 up to a correction of order
  sigma^2 / (1 - cos theta).
The cells draw independent proposals, so the mesh mean is within a few standard
errors (exact variances of the uniform cap and length variables) of these closed
forms.  Terms whose interaction is off are exactly zero."""
import math

import numpy as np

import oracle as O
import workloads as W

KB = 1.380649e-23


def uniform_state(n, m0):
    m = np.zeros((n, 3))
    m[:, 0] = m0
    return m


def test_exchange_term_closed_form():
    n = 256
    h = 5e-9
    spec = W._base((n, n, 1), (h, h, h), pbc=(True, True, False), A0=1.3e-11, T=300.0, Tc=870.0)
    o = O.Oracle(spec)
    m0 = 0.9
    theta = 30.0
    out = o.trial_terms(uniform_state(n * n, m0), None, 7, 0, 5, theta)
    kT = KB * 300.0
    cex = h ** 3 * 1.3e-11 / h ** 2 / kT
    sig = o.tables()["sigma"][0]
    a = 1.0 - math.cos(math.radians(theta))
    want = 4 * cex * m0 ** 2 * (sig ** 2 / 3 + a)
    # per cell 4 cex m0^2 ((s-1)^2 + 2 s t): dominated by 2 t, t uniform on [0, a]
    se = 4 * cex * m0 ** 2 * 2 * a / math.sqrt(12 * n * n)
    assert abs(out[0] - want) < 5 * se, (out[0], want, se)
    assert out[1] == 0.0 and out[2] == 0.0 and out[3] == 0.0 and out[5] == 0.0
    assert out[4] > 0.0                               # the longitudinal term is always there


def test_zeeman_term_closed_form():
    n = 256
    h = 5e-9
    B = 0.1
    spec = W._base((n, n, 1), (h, h, h), A0=0.0, B=(B, 0.0, 0.0), T=300.0, Tc=870.0)
    o = O.Oracle(spec)
    m0 = 0.85
    theta = 40.0
    out = o.trial_terms(uniform_state(n * n, m0), None, 3, 1, 11, theta)
    kT = KB * 300.0
    z = h ** 3 * spec["Ms0"] * B * m0 / kT
    a = 1.0 - math.cos(math.radians(theta))
    sig = o.tables()["sigma"][0]
    want = z * a / 2
    se = z * a / math.sqrt(12 * n * n)
    assert abs(out[3] - want) < 5 * se + z * sig ** 2 / a, (out[3], want, se)
    assert out[0] == 0.0 and out[1] == 0.0 and out[2] == 0.0 and out[5] == 0.0


def test_terms_follow_their_interactions():
    # DMI, anisotropy and demag switched on one at a time give a positive term
    base = dict(A0=0.0, T=300.0, Tc=700.0)
    mesh, h = (24, 20, 1), (3e-9, 3e-9, 2e-9)
    m = W.random_state(24 * 20, 4, 0.7, 0.9)[:, :3].astype(np.float64)
    for key, extra, idx in (("dmi", {"D0": 1.5e-3}, 1), ("an", {"K1": 3e5}, 2), ("demag", {"demag": True}, 5)):
        o = O.Oracle(W._base(mesh, h, **base, **extra))
        out = o.trial_terms(m, None, 2, 0, 9, 25.0)
        assert out[idx] > 0.0, key
        for k in (0, 1, 2, 3, 5):
            if k != idx:
                assert out[k] == 0.0, (key, k, out)
