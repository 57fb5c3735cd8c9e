"""Oracle pins of the zero-temperature steepest-descent minimizer (the paper's
SDesc comparison method, Sec. III), CPU only.

- Stoner-Wohlfarth: a single cubic cell with uniaxial anisotropy K(T) along z
  in a field at angle psi from z settles at the angle theta that solves
  K(T) sin 2 theta = Ms0 m_e B sin(psi - theta) (the isotropic self-demag of a
  cube exerts no torque); root found here by bisection.
- An open film with exchange and an in-plane field along x only (no demag, no
  anisotropy): the minimum is the uniform state along the field, reached from
  a tilted, noisy start.
- The returned state has |m| = m_e in every cell and the torque criterion met.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


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


@pytest.mark.parametrize("psi_deg,B", [(30.0, 0.02), (60.0, 0.05), (80.0, 0.01)])
def test_stoner_wohlfarth_angle(psi_deg, B):
    psi = math.radians(psi_deg)
    K1, Ms0, T, Tc = 5e4, 8e5, 300.0, 870.0
    s = W._base((1, 1, 1), (5e-9, 5e-9, 5e-9), Ms0=Ms0, K1=K1, T=T, Tc=Tc, demag=True,
                B=(B * math.sin(psi), 0.0, B * math.cos(psi)))
    o = O.Oracle(s)
    me = O.me(T, Tc)
    KT = K1 * me ** 3
    theta = _bisect(lambda t: KT * math.sin(2 * t) - Ms0 * me * B * math.sin(psi - t), 0.0, psi)
    m0 = np.array([[0.0, 0.0, me]])
    m, ok, it, tq = o.sdesc(m0, maxit=5000, tol=1e-10)
    assert ok, (it, tq)
    got = math.atan2(m[0, 0], m[0, 2])
    assert abs(m[0, 1]) < 1e-14
    assert got == pytest.approx(theta, abs=1e-9)
    assert np.linalg.norm(m[0]) == pytest.approx(me, rel=1e-14)


def test_film_in_field_aligns_with_the_field():
    s = W._base((8, 8, 1), (4e-9, 4e-9, 4e-9), B=(0.05, 0.0, 0.0), demag=False)
    o = O.Oracle(s)
    me = O.me(300.0, 870.0)
    rng = np.random.default_rng(2)
    m0 = np.tile([0.6, 0.5, 0.3], (64, 1)) + 0.05 * rng.standard_normal((64, 3))
    m, ok, it, tq = o.sdesc(m0, maxit=20000, tol=1e-8)
    assert ok, (it, tq)
    assert np.abs(m[:, 0] - me).max() < 1e-12
    assert np.abs(m[:, 1:]).max() < 1e-6
    assert np.allclose(np.linalg.norm(m, axis=1), me, rtol=1e-14)


def test_torque_criterion_and_energy_decrease():
    s = W._base((10, 6, 1), (3e-9, 3e-9, 2e-9), A0=1.2e-11, D0=1e-3, K1=3e5, Tc=650.0, T=300.0,
                Ms0=7e5, B=(0.02, 0.01, 0.05), demag=True)
    o = O.Oracle(s)
    m0 = W.smooth_state(s["mesh"], 3, 0.8)[:, :3].astype(np.float64)
    e0 = o.energy(m0 / np.linalg.norm(m0, axis=1, keepdims=True) * O.me(300.0, 650.0))[0]
    m, ok, it, tq = o.sdesc(m0, maxit=20000, tol=1e-6)
    assert ok and tq < 1e-6
    assert o.energy(m)[0] < e0
    # the torque of the result, recomputed from the gradient
    G, _, _ = o.energy_grad(m)
    u = m / np.linalg.norm(m, axis=1, keepdims=True)
    t = np.linalg.norm(np.cross(u, G), axis=1) / np.linalg.norm(G, axis=1)
    assert t.max() < 1e-6
