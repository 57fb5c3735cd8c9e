"""GPU tests of the float-float demag convolution (mmc_options.demag_fp64 = 2,
Sec. III, Eq. 14): the FFT convolution of the sweep's field carried in pairs of
FP32 values on the FP32 pipe.

- The field equals the oracle's FP64 field to 1e-10 of its largest entry (the
  FP32 convolution is ~1e-6 off) on square, ragged, periodic (circular), 3D and
  per-cell (granular) chains, alone and mixed in one batch.
- One sublattice pass with that field agrees with the oracle cell by cell within
  the FP32 sweep's bound, its decision values as close to the oracle's as with
  the FP64 convolution.
- Whole iterations with the float-float field and with the FP64 field from the
  same state end equal except the few cells whose FP32 field rounds differently.
"""
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
    "periodic256": [W.chiral_periodic(256, 300.0, 4)],
    "film3d": [W._base((24, 20, 4), (3e-9, 3e-9, 2e-9), demag=True, Ms0=8e5)],
    "granular": [W.granular_chain(200, 3, demag=True)],
    "mixed": [_chiral(512, 512, 100.0), _chiral(200, 130, 590.0), W.chiral_periodic(128, 200.0, 3),
              W.granular_chain(150, 4, demag=True)],
}


@pytest.mark.parametrize("name", list(CASES))
def test_ff_field_matches_oracle(P, name):
    specs = CASES[name]
    gff = P.MMC(specs, demag=1, demag_fp64=2)
    g32 = P.MMC(specs, demag=1, demag_fp64=0)
    for k, sp in enumerate(specs):
        n = int(np.prod(sp["mesh"]))
        m4 = W.random_state(n, 31 + k, 0.3, 0.9)
        for g in (gff, g32):
            g.set_m(m4, k)
        Ho = O.Oracle(sp).demag_field(m4[:, :3].astype(np.float64), "fft")
        scale = np.abs(Ho).max()
        eff = np.abs(gff.sweep_field(k) - Ho).max() / scale
        e32 = np.abs(g32.sweep_field(k) - Ho).max() / scale
        print("%s chain %d %s: float-float %.2e, FP32 %.2e (of max |H|)" % (name, k, sp["mesh"], eff, e32))
        assert eff < 1e-10 and eff < 1e-3 * e32


def test_ff_one_pass_matches_oracle(P):
    """One red and one black pass of a ragged chiral chain with the float-float
    field against the oracle's pass with its FP64 field."""
    spec = _chiral(301, 263, 200.0)
    n = 301 * 263
    m4 = W.smooth_state(spec["mesh"], 6, 0.9, tilt=0.8)
    g = P.MMC(spec, demag=1, demag_fp64=2)
    o = O.Oracle(spec)
    H = o.demag_field(m4[:, :3].astype(np.float64), "fft")
    for color in (0, 1):
        g.set_m(m4)
        dec, acc = g.pass_debug(0, color, 3, 41, 25.0)
        _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 3, 0, 41, 25.0, H=H, o=o)
        print("ff pass", color, compare_pass(dec, acc, dec_o, acc_o, band_o, wsum=exchange_weight_sum(spec)))


def test_ff_iterations_agree_with_fp64(P):
    """Three iterations of a mixed batch with the float-float and with the FP64
    convolution from the same states: the sweep sees both fields rounded to
    FP32, so every cell ends equal except the few whose field rounds the other
    way or whose decision then flips."""
    specs = CASES["mixed"]
    out = []
    for prec in (2, 1):
        g = P.MMC(specs, demag=1, demag_fp64=prec, adapt=0)
        for k, sp in enumerate(specs):
            g.set_m(W.random_state(int(np.prod(sp["mesh"])), 80 + k, 0.3, 0.9), k)
        g.sweep(3, 12)
        out.append([g.get_m(k) for k in range(len(specs))])
    for k, sp in enumerate(specs):
        d = np.abs(out[0][k][:, :3].astype(np.float64) - out[1][k][:, :3]).max(axis=1)
        nd = int((d > 1e-5).sum())
        print("ff vs fp64 chain", k, sp["mesh"], "differing", nd, "max |dm| elsewhere %.2e" % d[d <= 1e-5].max())
        assert nd <= 3 and d[d <= 1e-5].max() < 1e-6
