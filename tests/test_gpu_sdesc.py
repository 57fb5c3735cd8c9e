"""GPU tests of the zero-temperature steepest-descent minimizer (the paper's
SDesc comparison method, Sec. III) against closed forms and the oracle."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def _bisect(f, a, b, n=200):
    fa = f(a)
    for _ in range(n):
        c = 0.5 * (a + b)
        fc = f(c)
        if (fc < 0) == (fa < 0):
            a, fa = c, fc
        else:
            b = c
    return 0.5 * (a + b)


def test_stoner_wohlfarth_angle(P):
    """Single cubic cell, uniaxial K(T) along z, field at 60 deg from z: the
    angle solves K(T) sin 2 theta = Ms0 m_e B sin(psi - theta)."""
    psi, B, K1, Ms0, T, Tc = math.radians(60.0), 0.05, 5e4, 8e5, 300.0, 870.0
    s = W._base((1, 1, 1), (5e-9, 5e-9, 5e-9), Ms0=Ms0, K1=K1, T=T, Tc=Tc,
                B=(B * math.sin(psi), 0.0, B * math.cos(psi)))
    me = O.me(T, Tc)
    theta = _bisect(lambda t: K1 * me ** 3 * math.sin(2 * t) - Ms0 * me * B * math.sin(psi - t), 0.0, psi)
    g = P.MMC(s, demag=1)
    g.set_m(np.array([[0.0, 0.0, me, 0.0]], dtype=np.float32))
    r = g.minimize(0, maxit=5000, tol=1e-10)
    assert r["converged"], r
    m = g.get_m()[0]
    assert math.atan2(m[0], m[2]) == pytest.approx(theta, abs=2e-7)     # FP32 state
    assert np.linalg.norm(m[:3]) == pytest.approx(me, rel=1e-6)


@pytest.mark.parametrize("demag", [0, 1])
def test_film_matches_oracle(P, demag):
    """A film with exchange, DMI, anisotropy, field (and demag): the GPU and
    the oracle minimize from the same state to the same minimum."""
    s = W._base((10, 6, 1), (3e-9, 3e-9, 2e-9), A0=1.2e-11, D0=1e-3, K1=3e5, Tc=650.0, T=300.0,
                Ms0=7e5, B=(0.02, 0.01, 0.05), demag=bool(demag))
    m4 = W.smooth_state(s["mesh"], 3, 0.8)
    g = P.MMC(s, demag=demag)
    g.set_m(m4)
    r = g.minimize(0, maxit=20000, tol=1e-7)
    assert r["converged"], r
    mo, ok, it, tq = O.Oracle(s).sdesc(m4[:, :3].astype(np.float64), maxit=20000, tol=1e-7)
    assert ok
    mg = g.get_m()[:, :3].astype(np.float64)
    eo = O.Oracle(s).energy(mo)
    print("SDesc film demag=%d: GPU %d steps, oracle %d steps, max |dm| %.2e, E %.10e vs %.10e"
          % (demag, r["iters"], it, np.abs(mg - mo).max(), r["energy"][0], eo[0]))
    assert np.abs(mg - mo).max() < 2e-5
    assert r["energy"][0] == pytest.approx(eo[0], rel=1e-9)


def test_step_limit_and_rejections(P):
    s = W._base((6, 4, 1), (3e-9, 3e-9, 3e-9), K1=3e5, B=(0.02, 0.0, 0.0))
    g = P.MMC(s)
    g.set_m(W.smooth_state(s["mesh"], 4, 0.8))
    r = g.minimize(0, maxit=3, tol=1e-12)
    assert r["iters"] == 3 and not r["converged"]
    hot = P.MMC(W._base((4, 4, 1), (3e-9, 3e-9, 3e-9), T=900.0, Tc=870.0))
    with pytest.raises(Exception):
        hot.minimize(0)
