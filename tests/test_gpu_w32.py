"""GPU tests of the warp-resident 1024-point demag kernels (FFT variant 4,
chains whose padded grid is 1024 x 1024, i.e. 257..512 cells per in-plane
axis): the FP32 field the sweep uses equals the oracle's FP64 demag field
(Sec. III, Eq. 14) to FP32 rounding of the transforms, as closely as the
interleaved radix-16 kernels do, on square, ragged and mixed batches (uniform
and per-cell chains); one sublattice pass agrees with the oracle cell by cell;
grids of other sizes fall back to variant 1."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import compare_pass, exchange_weight_sum, lib_or_skip, oracle_pass

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def _chiral(nx, ny, T=300.0):
    return W.chiral(nx, T) | {"mesh": (nx, ny, 1)}


CASES = {
    "square512": [_chiral(512, 512)],
    "ragged301x263": [_chiral(301, 263, 450.0)],
    "mixed": [_chiral(512, 512, 100.0), _chiral(300, 300, 590.0), _chiral(257, 511, 610.0)],
    "granular": [W.granular_chain(400, 2, demag=True), W.granular_chain(300, 5, demag=True)],
}


@pytest.mark.parametrize("name", list(CASES))
def test_w32_sweep_field_matches_oracle(P, name):
    specs = CASES[name]
    g4 = P.MMC(specs, demag=1, fft_variant=4)
    g1 = P.MMC(specs, demag=1, fft_variant=1)
    assert g4.fft_tuning()[0] == 4 and g1.fft_tuning()[0] == 1
    for k, sp in enumerate(specs):
        n = int(np.prod(sp["mesh"]))
        m4 = W.random_state(n, 17 + k, 0.3, 0.9)
        for g in (g4, g1):
            g.set_m(m4, k)
        Ho = O.Oracle(sp).demag_field(m4[:, :3].astype(np.float64), "fft")
        scale = np.abs(Ho).max()
        e4 = np.abs(g4.sweep_field(k) - Ho).max() / scale
        e1 = np.abs(g1.sweep_field(k) - Ho).max() / scale
        print("%s chain %d %s: warp 32x32 %.2e, radix 16 %.2e (of max |H|)" % (name, k, sp["mesh"], e4, e1))
        assert e4 < 5e-6 and e4 < 3.0 * e1 + 1e-7


def test_w32_one_pass_matches_oracle(P):
    """One red and one black pass of a 512 x 512 chiral chain with the demag
    field of the warp kernels against the oracle's pass with its FP64 field."""
    spec = _chiral(512, 512, 200.0)
    n = 512 * 512
    m4 = W.smooth_state(spec["mesh"], 6, 0.9, tilt=0.8)
    g = P.MMC(spec, demag=1, fft_variant=4)
    o = O.Oracle(spec)
    H = o.demag_field(m4[:, :3].astype(np.float64), "fft")
    for color in (0, 1):
        g.set_m(m4)
        dec, acc = g.pass_debug(0, color, 3, 41, 25.0)
        _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 3, 0, 41, 25.0, H=H, o=o)
        print("w32 pass", color, compare_pass(dec, acc, dec_o, acc_o, band_o, wsum=exchange_weight_sum(spec)))


def test_w32_falls_back_off_its_grids(P):
    """Variant 4 on grids it does not handle (a 256 x 256 chain, padded 512;
    a periodic 512 x 512 chain, transformed circularly) runs variant 1."""
    for specs in ([W.chiral(256, 300.0)], [W.chiral_periodic(512, 300.0, 2)], [_chiral(512, 512), W.chiral(200)]):
        g = P.MMC(specs, demag=1, fft_variant=4)
        assert g.fft_tuning()[0] == 1


def _ndiff(a, b):
    d = np.abs(a[:, :3].astype(np.float64) - b[:, :3]).max(axis=1)
    return int((d > 1e-5).sum()), float(d[d <= 1e-5].max(initial=0.0))


def test_fused_black_pass_agrees_with_separate_kernels(P):
    """The black pass fused with the next forward row transforms (default on
    this path) against separate kernels: three iterations of a batch of square,
    ragged and periodic chains from the same states end equal to FP32 rounding
    except the few cells a decision within that rounding of zero can flip; the
    per-kernel timing reports the fused kernel."""
    specs = [_chiral(512, 512, 120.0), _chiral(301, 263, 590.0),
             _chiral(400, 300, 450.0) | {"pbc": (True, True, False)}]
    out = []
    for fuse in (1, 0):
        g = P.MMC(specs, demag=1, fft_variant=4, fuse_passes=fuse, adapt=0)
        for k, sp in enumerate(specs):
            g.set_m(W.random_state(int(np.prod(sp["mesh"])), 60 + k, 0.3, 0.9), k)
        g.sweep(3, 8)
        out.append([g.get_m(k) for k in range(len(specs))])
        ph = g.phase_times(2, 9)
        assert (ph["black_pass_rows_fwd"][1] > 0) == (fuse == 1)
    for k in range(len(specs)):
        nd, agree = _ndiff(out[0][k], out[1][k])
        print("fused vs separate chain", k, specs[k]["mesh"], "differing", nd, "max |dm| elsewhere %.2e" % agree)
        assert nd <= 2 and agree < 1e-6


def test_fused_path_matches_oracle(P):
    """Three whole iterations of a ragged chain on the fused path against the
    oracle's run from the same state."""
    spec = _chiral(301, 263, 520.0)
    n = 301 * 263
    m4 = W.random_state(n, 71, 0.3, 0.6)
    g = P.MMC(spec, demag=1, fft_variant=4, adapt=0)
    g.set_m(m4)
    g.sweep(3, 5)
    o = O.Oracle(spec)
    st = O.new_state(seed=5, chain=0, theta_deg=30.0, adapt=False, demag_mode=1)
    mo, _, _ = o.run(m4[:, :3].astype(np.float64), 3, st)
    nd, agree = _ndiff(g.get_m(0), mo)
    print("fused path vs oracle: differing", nd, "max |dm| elsewhere %.2e" % agree)
    assert nd <= 4 and agree < 1e-5
