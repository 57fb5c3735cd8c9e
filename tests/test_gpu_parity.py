"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

- thermodynamic tables (Eqs. 8, 9, 13): 1e-12 relative
- one sublattice pass (Sec. II, Eq. 5): accept bits identical except where the
  oracle's decision value lies inside the FP32 error bound of the GPU's value;
  decision values within that bound.  Meshes span several blocks and ragged
  tails: periodic 32x32, odd open 33x31, 4x4x1, 3D 9x6x4 with DMI and
  anisotropy, the 256x256 demag film, a batch of uneven chains, granular
  per-cell material.
- demag field (Eq. 14, FP64 convolution) and energy terms vs the oracle
- observables: |m| histogram equal to the oracle's FP64 binning except cells
  within FP32 rounding of a bin edge, moments to FP64 rounding
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import compare_hist, compare_pass, lib_or_skip, oracle_pass

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def full_spec(mesh, demag=False, pbc=(False, False, False), seed=0):
    return W._base(mesh, (3e-9, 3e-9, 2e-9), pbc=pbc, A0=1.2e-11, D0=1.1e-3, K1=3e5,
                   K2=2e4, eA=(0.3, 0.2, 0.93), Tc=650.0, T=330.0, Ms0=7e5,
                   B=(0.02, -0.01, 0.05), demag=demag)


def test_tables_match_oracle(P):
    for T, Tc in [(300, 870), (800, 870), (869.5, 870), (869.99, 870), (900, 870), (50, 600), (610, 600)]:
        s = W._base((4, 2, 1), (4e-9, 4e-9, 4e-9), T=T, Tc=Tc)
        g = P.MMC(s).tables()
        o = O.Oracle(s).tables()
        # Eq. 8 divides by 1 - 3 B'(x) Tc / T, which vanishes at Tc: rounding is
        # amplified by about 1 / |1 - T/Tc| there
        rel = 1e-12 + 1e-15 / abs(1.0 - T / Tc)
        for k in ("me", "chi", "sigma"):
            assert g[k][0] == pytest.approx(o[k][0], rel=rel, abs=1e-300), (T, Tc, k)


CASES = {
    "permalloy32": (W.permalloy32(), 0),
    "odd33x31": (W._base((33, 31, 1), (5e-9, 5e-9, 5e-9), B=(0.01, 0.0, 0.0)), 0),
    "tiny4x4": (full_spec((4, 4, 1), pbc=(True, True, False)), 0),
    "full3d": (full_spec((9, 6, 4)), 0),
    "periodic3d": (full_spec((8, 6, 4), pbc=(True, True, True)), 0),
    "cubic": (full_spec((12, 10, 2)) | {"aniso": "cubic", "K1": 4.8e5, "K2": -1e5}, 0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_one_pass_matches_oracle(P, name):
    spec, _ = CASES[name]
    n = int(np.prod(spec["mesh"]))
    m4 = W.random_state(n, 21, 0.75, 0.95)
    g = P.MMC(spec)
    for color in (0, 1):
        for sweep, theta in ((0, 30.0), (17, 5.0), (123456, 120.0)):
            g.set_m(m4)       # the diagnostic pass updates the state: restart from m4
            dec_g, acc_g = g.pass_debug(0, color, sweep, 11, theta)
            _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, sweep, 0, 11, theta)
            stats = compare_pass(dec_g, acc_g, dec_o, acc_o, band_o)
            print(name, color, sweep, stats)


def test_one_pass_with_demag_film(P):
    spec = W.film256(128, B_mT=20.0)
    n = 128 * 128
    m4 = W.smooth_state(spec["mesh"], 3, 0.86)
    for fp64, cufft in ((0, 0), (1, 0), (0, 1), (1, 1)):
        g = P.MMC(spec, demag=1, demag_fp64=fp64, demag_cufft=cufft)
        o = O.Oracle(spec)
        H = o.demag_field(m4[:, :3].astype(np.float64), "fft")
        for color in (0, 1):
            g.set_m(m4)
            dec_g, acc_g = g.pass_debug(0, color, 5, 3, 25.0)
            _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 5, 0, 3, 25.0, H=H)
            print("film128 fp64=%d cufft=%d" % (fp64, cufft), color,
                  compare_pass(dec_g, acc_g, dec_o, acc_o, band_o))


def test_demag_field_fp64(P):
    for mesh, h in (((48, 40, 1), (4e-9, 4e-9, 4e-9)), ((16, 12, 4), (3e-9, 2e-9, 2.5e-9)),
                    ((256, 192, 1), (4e-9, 4e-9, 4e-9)), ((130, 3, 1), (2e-9, 2e-9, 1e-9)),
                    ((1, 1, 1), (5e-9, 5e-9, 5e-9)), ((7, 1, 1), (2e-9, 3e-9, 4e-9))):
        n = int(np.prod(mesh))
        spec = W._base(mesh, h, demag=True, Ms0=6e5)
        m4 = W.random_state(n, 5, 0.5, 1.0)
        g = P.MMC(spec, demag=1)
        g.set_m(m4)
        Hg = g.demag_field(0)
        Ho = O.Oracle(spec).demag_field(m4[:, :3].astype(np.float64), "direct" if n <= 4096 else "fft")
        scale = np.abs(Ho).max()
        print("demag fp64", mesh, np.abs(Hg - Ho).max() / scale)
        assert np.abs(Hg - Ho).max() < 1e-9 * scale, (mesh, np.abs(Hg - Ho).max() / scale)


def test_energy_terms(P):
    for spec in (full_spec((9, 6, 4), demag=True), full_spec((8, 6, 1), pbc=(True, True, False)),
                 W.chiral(32, 610.0), W.energy3d(16, 4)):
        n = int(np.prod(spec["mesh"]))
        m4 = W.random_state(n, 9, 0.3, 0.9)
        g = P.MMC(spec, demag=int(spec["demag"]))
        g.set_m(m4)
        Eg = g.energy(0)
        Eo = O.Oracle(spec).energy(m4[:, :3].astype(np.float64))
        scale = np.abs(Eo[1:]).sum()
        for k in range(7):
            assert Eg[k] == pytest.approx(Eo[k], abs=1e-9 * scale), (spec["mesh"], k, Eg, Eo)


def test_observables_current_state(P):
    spec = W._base((37, 29, 2), (5e-9, 5e-9, 5e-9))
    n = 37 * 29 * 2
    m4 = W.random_state(n, 4, 0.2, 1.05)
    g = P.MMC(spec)
    g.set_m(m4)
    ob = g.observables(0)
    assert compare_hist(ob["hist"], m4, 200, 1.0) <= 2      # cells within FP32 rounding of an edge
    v = m4[:, :3].astype(np.float64)
    L = np.linalg.norm(v, axis=1)
    assert ob["mean_m"] == pytest.approx(v.mean(0), rel=1e-12, abs=1e-15)
    assert ob["mean_len"] == pytest.approx(L.mean(), rel=1e-12)
    assert ob["mean_len2"] == pytest.approx((L * L).mean(), rel=1e-12)
    assert ob["nsnap"] == 0 and ob["nonfinite"] == 0


def test_batch_of_uneven_chains(P):
    specs = [full_spec((9, 6, 4)), W.permalloy32(), W._base((33, 31, 1), (5e-9,) * 3),
             W.chiral(24, 610.0) | {"demag": False}]
    g = P.MMC(specs)
    states = []
    for k, sp in enumerate(specs):
        n = int(np.prod(sp["mesh"]))
        states.append(W.random_state(n, 30 + k, 0.7, 0.9))
        g.set_m(states[-1], k)
    for k, sp in enumerate(specs):
        for color in (0, 1):
            g.set_m(states[k], k)
            dec_g, acc_g = g.pass_debug(k, color, 7, 99, 40.0)
            _, acc_o, dec_o, band_o = oracle_pass(sp, states[k], color, 7, k, 99, 40.0)
            compare_pass(dec_g, acc_g, dec_o, acc_o, band_o)


def test_granular_per_cell_chain(P):
    spec = W.granular_chain(48, 3, demag=False)
    spec["B"] = (0.0, 0.0, 0.05)
    n = 48 * 48
    m4 = W.random_state(n, 8, 0.6, 0.9)
    g = P.MMC(spec)
    for color in (0, 1):
        g.set_m(m4)
        dec_g, acc_g = g.pass_debug(0, color, 2, 5, 30.0)
        _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 2, 0, 5, 30.0)
        print("granular", color, compare_pass(dec_g, acc_g, dec_o, acc_o, band_o))


def test_mixed_batch_of_uniform_and_per_cell_chains(P):
    """A batch mixing uniform chains with a per-cell granular chain: every chain
    of the batch is read through per-cell tables (one launch treats all chains
    alike); each chain's pass still agrees with the oracle."""
    specs = [W.permalloy32(), W.granular_chain(40, 4, demag=False), full_spec((9, 6, 4))]
    g = P.MMC(specs)
    for k, sp in enumerate(specs):
        n = int(np.prod(sp["mesh"]))
        m4 = W.random_state(n, 40 + k, 0.6, 0.9)
        for color in (0, 1):
            g.set_m(m4, k)
            dec_g, acc_g = g.pass_debug(k, color, 4, 77, 35.0)
            _, acc_o, dec_o, band_o = oracle_pass(sp, m4, color, 4, k, 77, 35.0)
            compare_pass(dec_g, acc_g, dec_o, acc_o, band_o)


def test_pass_updates_exactly_the_accepted_cells(P):
    spec, _ = CASES["full3d"]
    n = int(np.prod(spec["mesh"]))
    m4 = W.random_state(n, 22, 0.75, 0.95)
    g = P.MMC(spec)
    g.set_m(m4)
    dec, acc = g.pass_debug(0, 1, 3, 8, 35.0)
    m1 = g.get_m()
    m_o, acc_o, dec_o, band_o = oracle_pass(spec, m4, 1, 3, 0, 8, 35.0)
    compare_pass(dec, acc, dec_o, acc_o, band_o)
    moved = np.any(m1[:, :3] != m4[:, :3], axis=1)
    assert np.array_equal(moved, acc == 1)
    # accepted vectors equal the oracle's FP64 proposals to FP32 rounding
    sel = acc == 1
    assert np.abs(m1[sel, :3] - m_o[sel]).max() < 4e-7


@pytest.mark.parametrize("per_pass", [0, 1])
def test_full_iterations_match_oracle(P, per_pass):
    """Whole iterations (demag, red, [demag], black) through mmc_sweep against the
    oracle's run loop (Eq. 14 frozen field once per iteration, or before each pass):
    every cell ends equal to FP32 rounding unless a decision sits inside the bound."""
    spec = W.film256(96, B_mT=20.0)
    spec["D0"] = 1e-3
    n = 96 * 96
    m4 = W.smooth_state(spec["mesh"], 5, 0.86)
    g = P.MMC(spec, demag=1, demag_per_pass=per_pass, adapt=0, theta0_deg=25.0)
    g.set_m(m4)
    g.sweep(3, 13)
    mg = g.get_m()[:, :3].astype(np.float64)
    o = O.Oracle(spec)
    st = O.new_state(seed=13, chain=0, theta_deg=25.0, adapt=False, demag_mode=2 if per_pass else 1)
    mo, _, _ = o.run(m4[:, :3].astype(np.float64), 3, st)
    d = np.abs(mg - mo).max(axis=1)
    differ = int((d > 1e-5).sum())
    print("full iterations per_pass=%d: max |dm| over agreeing cells %.2e, differing cells %d"
          % (per_pass, d[d <= 1e-5].max(), differ))
    assert differ <= 2          # a flipped decision inside the FP32 bound changes a cell and its neighbours later


@pytest.mark.parametrize("mesh,bins,lo,hi", [((48, 40, 1), 100, 0.0, np.pi), ((12, 10, 6), 37, 0.1, 1.2)])
def test_angle_hist_matches_oracle(P, mesh, bins, lo, hi):
    """Angular-deviation histogram (Sec. II, Fig. 1d-f) of one chain of a batch
    equals the oracle's on the same state, count for count."""
    spec = W._base(mesh, (3e-9,) * 3)
    n = int(np.prod(mesh))
    m4 = W.smooth_state(mesh, 9, 0.8, tilt=0.9)
    g = P.MMC([W.permalloy32(8), spec])
    g.set_m(m4, 1)
    h, d = g.angle_hist(1, bins, lo, hi)
    ho, do = O.Oracle(spec).angle_hist(m4[:, :3].astype(np.float64), bins, lo, hi)
    assert np.allclose(d, do, rtol=0, atol=1e-14)
    assert h.sum() == n
    assert np.array_equal(h, ho)


@pytest.mark.parametrize("mesh", [(2048, 6, 1), (6, 2048, 1), (2048, 4, 2)])
def test_longest_transforms(P, mesh):
    """Meshes whose padded length is the largest supported (4096) along x, along
    y, and in 3D: FP64 field against the oracle, and one pass with each FP32
    kernel variant (a variant that cannot hold a 4096-point row falls back)."""
    n = int(np.prod(mesh))
    spec = W._base(mesh, (2e-9, 2e-9, 2e-9), demag=True, Ms0=6e5, A0=1e-11, B=(0.01, 0.0, 0.0))
    m4 = W.smooth_state(mesh, 2, 0.85)
    o = O.Oracle(spec)
    Ho = o.demag_field(m4[:, :3].astype(np.float64), "fft")
    g = P.MMC(spec, demag=1)
    g.set_m(m4)
    err = np.abs(g.demag_field(0) - Ho).max() / np.abs(Ho).max()
    print("longest transforms", mesh, err)
    assert err < 1e-9
    for variant in (1, 2, 3):
        gv = P.MMC(spec, demag=1, fft_variant=variant)
        for color in (0, 1):
            gv.set_m(m4)
            dec_g, acc_g = gv.pass_debug(0, color, 1, 4, 20.0)
            _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 1, 0, 4, 20.0, H=Ho, o=o)
            compare_pass(dec_g, acc_g, dec_o, acc_o, band_o)
