"""GPU chains against exact equilibrium laws (the laws the oracle is pinned by in
tests/test_oracle_mc.py), through the C ABI: an open chain coupled by exchange
(the classical Heisenberg chain's bond law), two cells with exchange and DMI
(the conditional von Mises-Fisher law of the pair energy) and free cells with
uniaxial anisotropy (exp(kappa c^2)).  Each statistic has mean zero exactly."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu

KB = O.KB


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def _block_stats(vals, nblocks):
    b = np.asarray(vals).reshape(nblocks, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nblocks)


def _trap(yv, xv):
    return float(np.sum((yv[1:] + yv[:-1]) * np.diff(xv)) / 2.0)


def _lang(k):
    return 1.0 / np.tanh(k) - 1.0 / k


def test_exchange_chain_bond_law(P):
    T, Tc, A0, h = 300.0, 870.0, 1.3e-11, 0.4e-9
    n = 64
    spec = W._base((n, 1, 1), (h, h, h), A0=A0, Tc=Tc, T=T)
    me = O.me(T, Tc)
    c_kt = h * A0 / (KB * T)
    g = P.MMC(spec, adapt=0, theta0_deg=60.0)
    g.set_m(W.random_state(n, 11, me, me))
    g.sweep(500, 13)
    vals = []
    for _ in range(3000):
        g.sweep(5, 13)
        m = g.get_m(0)[:, :3].astype(np.float64)
        ln = np.linalg.norm(m, axis=1)
        u = m / ln[:, None]
        vals.append(np.mean(np.sum(u[:-1] * u[1:], axis=1) - _lang(2.0 * c_kt * ln[:-1] * ln[1:])))
    mean, se = _block_stats(vals, 30)
    print("exchange chain: %.4f +- %.4f" % (mean, se))
    assert se < 0.006 and abs(mean) < 4.0 * se + 1e-3


def test_two_cell_exchange_dmi_law(P):
    T, Tc, A0, h = 300.0, 870.0, 1.3e-11, 0.4e-9
    D0 = 2.0 * A0 / h
    spec = W._base((2, 1, 1), (h, h, h), A0=A0, D0=D0, Tc=Tc, T=T)
    me = O.me(T, Tc)
    c, d = h * A0, h * h * D0
    y = np.array([0.0, 1.0, 0.0])
    g = P.MMC(spec, adapt=0, theta0_deg=60.0)
    g.set_m(np.array([[me, 0.0, 0.0, 0.0], [0.0, me, 0.0, 0.0]], dtype=np.float32))
    g.sweep(200, 41)
    vals = []
    for _ in range(20000):
        g.sweep(2, 41)
        m = g.get_m(0)[:, :3].astype(np.float64)
        ln = np.linalg.norm(m, axis=1)
        u = m / ln[:, None]
        f = ln[0] * ln[1] / (KB * T)
        k0 = f * (2.0 * c * u[1] + d * np.cross(u[1], y))
        k1 = f * (2.0 * c * u[0] + d * np.cross(y, u[0]))
        n0, n1 = np.linalg.norm(k0), np.linalg.norm(k1)
        vals.append(0.5 * (u[0] @ k0 / n0 - _lang(n0) + u[1] @ k1 / n1 - _lang(n1)))
    mean, se = _block_stats(vals, 100)
    print("exchange + DMI pair: %.4f +- %.4f" % (mean, se))
    assert se < 0.006 and abs(mean) < 4.0 * se + 1e-3


def test_uniaxial_anisotropy_law(P):
    T, Tc, h = 300.0, 870.0, 5e-9
    V = h ** 3
    me = O.me(T, Tc)
    kappa = 2.0
    K1 = kappa * KB * T / (V * me ** 3)
    spec = W._base((64, 64, 1), (h, h, h), A0=0.0, K1=K1, eA=(0.0, 0.0, 1.0), Tc=Tc, T=T)
    g = P.MMC(spec, adapt=0, theta0_deg=60.0)
    g.set_m(W.random_state(64 * 64, 21, me, me))
    g.sweep(200, 23)
    vals = []
    for _ in range(200):
        g.sweep(3, 23)
        m = g.get_m(0)[:, :3].astype(np.float64)
        cz = m[:, 2] / np.linalg.norm(m, axis=1)
        vals.append(np.mean(cz * cz))
    mean, se = _block_stats(vals, 20)
    x = np.linspace(-1.0, 1.0, 200001)
    w = np.exp(kappa * x * x)
    ref = _trap(w * x * x, x) / _trap(w, x)
    print("uniaxial: %.4f +- %.4f (exact %.4f)" % (mean, se, ref))
    assert se < 0.003 and abs(mean - ref) < 4.0 * se + 5e-4
