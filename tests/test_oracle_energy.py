"""Oracle energy pins (CPU only).

- The pair energies equal half the per-vector sums of the paper's Eq. 10
  (exchange, discrete Laplacian), Eq. 15 (interfacial DMI, central differences)
  and Eq. 14 (demag) on lattices periodic in-plane: the paper's factor 2.
- Brute force: the local energy change of a trial move equals E(after) -
  E(before) of the full energy, all terms, per-cell material, grains; with the
  frozen demag field the gap is exactly the self term (Eq. 14 reading).
- Analytic gradient vs central differences of the full energy; parameter
  gradients vs differences in the parameters.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _rand_m(n, seed, lo=0.5, hi=1.0):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * rng.uniform(lo, hi, (n, 1))


def _full_spec(mesh, pbc, demag, seed=0, cubic=False, grains=True, T=350.0):
    rng = np.random.default_rng(100 + seed)
    n = mesh[0] * mesh[1] * mesh[2]
    e = rng.standard_normal((n, 3))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    s = W._base(mesh, (3e-9, 4e-9, 2.5e-9), pbc=pbc, A0=1.1e-11, D0=-2.2e-3,
                Ms0=rng.uniform(5e5, 9e5, n), K1=rng.uniform(1e5, 6e5, n),
                K2=rng.uniform(-5e4, 5e4, n), eA=e, Tc=rng.uniform(550, 700, n),
                T=rng.uniform(0.5, 1.3, n) * T, B=(0.02, -0.03, 0.05), demag=demag,
                grain=(rng.integers(0, 3, n) if grains else None), grain_exch_scale=0.3,
                aniso="cubic" if cubic else "uniaxial")
    return s


@pytest.mark.parametrize("mesh", [(8, 6, 1), (4, 4, 1)])
def test_pair_energies_are_half_of_pervector_sums(mesh):
    s = W._base(mesh, (3e-9, 4e-9, 2.5e-9), pbc=(True, True, False), A0=1.3e-11,
                D0=1.7e-3, demag=True, Ms0=7e5)
    o = O.Oracle(s)
    m = _rand_m(o.n, 1)
    E = o.energy(m)
    pv = o.pervector_sums(m)
    assert pv[0] == pytest.approx(2.0 * E[1], rel=1e-12)      # Eq. 10
    assert pv[1] == pytest.approx(2.0 * E[2], rel=1e-12)      # Eq. 15
    assert pv[2] == pytest.approx(2.0 * E[6], rel=1e-12)      # Eq. 14


def test_dmi_sign_follows_eq15_for_a_cycloid():
    # a Neel cycloid m = (sin kx, 0, cos kx): Eq. 15 energy density
    # -2 D0 m.(z div m - grad m_z) per vector = -2 D0 (cos*k cos + sin*k sin) = -2 D0 k
    nx = 16
    s = W._base((nx, 2, 1), (2e-9, 2e-9, 1e-9), pbc=(True, True, False), A0=0.0, D0=1.5e-3)
    o = O.Oracle(s)
    k = 2 * np.pi / nx
    x = np.arange(nx * 2) % nx
    m = np.stack([np.sin(k * x), 0 * x, np.cos(k * x)], axis=1)
    E = o.energy(m)[2]
    V = 4e-27
    # central-difference wavenumber sin(k h)/h replaces k on the lattice
    expected = -V * 1.5e-3 * np.sin(k) / 2e-9 * (nx * 2)
    assert E == pytest.approx(expected, rel=1e-12)
    assert E < 0          # positive D0 favours this rotation sense


@pytest.mark.parametrize("case", [
    dict(mesh=(4, 4, 1), pbc=(True, True, False), demag=True),
    dict(mesh=(4, 4, 1), pbc=(False, False, False), demag=True),
    dict(mesh=(3, 3, 2), pbc=(False, False, False), demag=True),
    dict(mesh=(4, 2, 2), pbc=(True, True, False), demag=False, cubic=True),
    dict(mesh=(5, 3, 1), pbc=(False, False, False), demag=False, T=700.0),
])
def test_local_energy_change_brute_force(case):
    cubic = case.pop("cubic", False)
    T = case.pop("T", 350.0)
    s = _full_spec(case["mesh"], case["pbc"], case["demag"], cubic=cubic, T=T)
    o_exact = O.Oracle(s, demag_self=True)
    o_frozen = O.Oracle(s, demag_self=False)
    rng = np.random.default_rng(5)
    m = _rand_m(o_exact.n, 7)
    H = o_exact.demag_field(m) if s["demag"] else np.zeros((o_exact.n, 3))
    E0 = o_exact.energy(m)
    self_t = O.newell(s["h"], (0, 0, 0))
    N = np.array([[self_t[0], self_t[3], self_t[4]], [self_t[3], self_t[1], self_t[5]],
                  [self_t[4], self_t[5], self_t[2]]])
    V = s["h"][0] * s["h"][1] * s["h"][2]
    for trial in range(12):
        i = int(rng.integers(0, o_exact.n))
        mn = m[i] + 0.3 * rng.standard_normal(3)
        m2 = m.copy()
        m2[i] = mn
        E1 = o_exact.energy(m2)
        dF = o_exact.local_dF(m, H, i, mn)
        scale = np.abs(E1[1:]).sum() + np.abs(E0[1:]).sum()
        assert dF[0] == pytest.approx(E1[0] - E0[0], abs=1e-11 * scale)
        for t in range(1, 6):
            assert dF[t] == pytest.approx(E1[t] - E0[t], abs=1e-11 * scale)
        # frozen-field demag (Eq. 14) = exact change minus the self term
        dfz = o_frozen.local_dF(m, H, i, mn)
        dM = s["Ms0"][i] * (mn - m[i])
        self_term = 0.5 * O.MU0 * V * dM @ N @ dM if s["demag"] else 0.0
        assert dfz[6] == pytest.approx(E1[6] - E0[6] - self_term, abs=1e-11 * scale)


@pytest.mark.parametrize("demag", [False, True])
def test_gradient_against_central_differences(demag):
    s = _full_spec((4, 3, 2), (False, False, False), demag, grains=False, T=300.0)
    o = O.Oracle(s)
    m = _rand_m(o.n, 11, 0.6, 0.9)
    g, _, _ = o.energy_grad(m)
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(10):
        i = int(rng.integers(0, o.n))
        a = int(rng.integers(0, 3))
        mp = m.copy(); mp[i, a] += h
        mm = m.copy(); mm[i, a] -= h
        fd = (o.energy(mp)[0] - o.energy(mm)[0]) / (2 * h)
        assert g[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g).max())


def test_parameter_gradients_against_differences():
    base = W._base((4, 4, 2), (4e-9, 4e-9, 4e-9), Ms0=6e5, A0=1e-11, D0=1.5e-3, K1=8e5,
                   Tc=600.0, T=300.0, demag=True, B=(0.01, 0.02, 0.03))
    m = _rand_m(32, 4, 0.7, 0.8)
    _, dp, E = O.Oracle(base).energy_grad(m)
    for k, key in enumerate(["Ms0", "A0", "D0", "K1"]):
        v = base[key]
        d = 1e-6 * v
        sp = dict(base); sp[key] = v + d
        sm = dict(base); sm[key] = v - d
        fd = (O.Oracle(sp).energy(m)[0] - O.Oracle(sm).energy(m)[0]) / (2 * d)
        assert dp[k] == pytest.approx(fd, rel=1e-6)
    # E_l is proportional to 1/chi (Eq. 7)
    tb = O.Oracle(base).tables()
    assert dp[4] == pytest.approx(-E[5] / tb["chi"][0], rel=1e-14)
