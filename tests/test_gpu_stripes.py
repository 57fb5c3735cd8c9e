"""Demag schedules finer than one update per pass (f-2): each sublattice pass in
S bands of rows with the demag field recomputed before every band.

- Whole iterations against the oracle's banded schedule (every cell equal to
  FP32 rounding unless a decision sits inside the FP32 bound).
- The band schedule with one stream and with chain groups on concurrent
  streams gives the same chains bit for bit (graph blocks and an eager tail).
- One band is the per-pass schedule; without demag the bands change nothing.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


@pytest.mark.parametrize("mesh,stripes", [((96, 96, 1), 4), ((40, 30, 1), 7), ((24, 20, 3), 5)])
def test_banded_iterations_match_oracle(P, mesh, stripes):
    spec = W._base(mesh, (4e-9, 4e-9, 4e-9), demag=True, A0=1.3e-11, D0=1e-3, B=(0.02, 0.0, 0.0))
    n = int(np.prod(mesh))
    m4 = W.smooth_state(mesh, 5, 0.86)
    g = P.MMC(spec, demag=1, demag_stripes=stripes, adapt=0, theta0_deg=25.0)
    g.set_m(m4)
    g.sweep(3, 13)
    mg = g.get_m()[:, :3].astype(np.float64)
    st = O.new_state(seed=13, chain=0, theta_deg=25.0, adapt=False, demag_mode=2, stripes=stripes)
    mo, _, _ = O.Oracle(spec).run(m4[:, :3].astype(np.float64), 3, st)
    d = np.abs(mg - mo).max(axis=1)
    differ = int((d > 1e-5).sum())
    print("bands %s S=%d: max |dm| over agreeing cells %.2e, differing cells %d"
          % (mesh, stripes, d[d <= 1e-5].max(), differ))
    assert differ <= 2


def test_bands_with_stream_groups_are_bitwise(P):
    specs = [W.chiral(40, 100.0 + 60.0 * k) for k in range(4)] + [W.film256(48)]
    out = []
    for groups in (1, 2):
        g = P.MMC(specs, demag=1, fft_variant=1, stream_groups=groups, demag_stripes=3)
        g.init_random(5)
        g.sweep(100, 5)
        g.sweep(23, 5)
        out.append([g.get_m(k) for k in range(len(specs))])
    for k in range(len(specs)):
        assert np.array_equal(out[0][k], out[1][k]), k


def test_one_band_and_no_demag(P):
    spec = W.film256(48, B_mT=20.0)
    a = P.MMC(spec, demag=1, demag_per_pass=1, fft_variant=1)
    b = P.MMC(spec, demag=1, demag_stripes=1, demag_per_pass=1, fft_variant=1)
    for g in (a, b):
        g.init_random(3)
        g.sweep(120, 3)
    assert np.array_equal(a.get_m(), b.get_m())
    nod = W.permalloy32(32)
    c = P.MMC(nod)
    d = P.MMC(nod, demag_stripes=6)
    for g in (c, d):
        g.init_random(4)
        g.sweep(120, 4)
    assert np.array_equal(c.get_m(), d.get_m())
    with pytest.raises(P.MmcError):
        P.MMC(spec, demag=1, demag_stripes=65)
