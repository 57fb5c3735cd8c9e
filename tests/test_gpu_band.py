"""GPU tests of the banded sublattice pass on shared-memory halo tiles
(mmc_options.sweep_tiles, Sec. II red-black decomposition): bands of rows
brought into shared memory by bulk asynchronous copies while the previous band
is computed.  It makes the same moves as the per-block pass: whole iterations
of both agree on batches of uneven, odd, periodic and demag chains;
its moves match the oracle cell by cell (one pass, ragged last bands); and a
wait for copies that never land gives up, skips its bands and is reported as
MMC_ERR_TIMEOUT without disturbing the GPU.  (It is compiled separately from
the per-block pass, so the two agree to FP32 rounding, not bit for bit; each
is deterministic on its own.)"""
import numpy as np
import pytest

import workloads as W
from gpu_common import compare_pass, exchange_weight_sum, lib_or_skip, oracle_pass

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def _mixed():
    return [W.chiral(64, 300.0), W.permalloy32(), W._base((33, 31, 1), (5e-9,) * 3, B=(0.0, 0.01, 0.0)),
            W.film256(96, 20.0) | {"mesh": (96, 80, 1)}, W.chiral(200, 590.0) | {"mesh": (200, 133, 1)},
            W.chiral_periodic(64, 150.0, 2)]


def test_band_pass_agrees_with_blockwise_pass(P):
    """Three whole iterations of a mixed batch (uneven, odd, periodic, demag
    chains) with the banded pass and with the per-block pass from the same
    state: the two kernels are compiled separately, so their energy terms round
    differently in the last bit, and every cell must end equal to FP32 rounding
    except the few a decision within that rounding of zero can flip."""
    specs = _mixed()
    out = []
    for tiles in (1, 0):
        g = P.MMC(specs, demag=1, fft_variant=1, sweep_tiles=tiles, adapt=0)
        for k, sp in enumerate(specs):
            g.set_m(W.random_state(int(np.prod(sp["mesh"])), 40 + k, 0.4, 0.9), k)
        g.sweep(3, 3)
        out.append([g.get_m(k) for k in range(len(specs))])
    for k, sp in enumerate(specs):
        d = np.abs(out[0][k][:, :3] - out[1][k][:, :3]).max(axis=1)
        ndiff = int((d > 1e-5).sum())
        print("chain", k, sp["mesh"], "max |dm| of agreeing cells %.2e, differing cells %d" % (d[d <= 1e-5].max(), ndiff))
        assert d[d <= 1e-5].max() < 1e-6 and ndiff <= 2


@pytest.mark.parametrize("mesh,pbc", [((200, 133, 1), (False, False, False)), ((64, 66, 1), (True, True, False)),
                                      ((1024, 9, 1), (False, False, False)), ((31, 7, 1), (False, False, False))])
def test_band_pass_matches_oracle(P, mesh, pbc):
    """One red and one black pass through the banded kernel against the oracle:
    rows per band 512 / hx with a ragged last band, periodic wrap of the halo
    rows and columns, the widest rows the banded pass takes (1024 cells)."""
    spec = W.chiral(64, 420.0) | {"mesh": mesh, "pbc": pbc}
    n = int(np.prod(mesh))
    m4 = W.random_state(n, 12, 0.3, 0.7)
    g = P.MMC(spec, demag=1, sweep_tiles=1)
    for color in (0, 1):
        g.set_m(m4)
        dec, acc = g.pass_debug(0, color, 6, 23, 35.0)
        _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 6, 0, 23, 35.0)
        print("band pass", mesh, pbc, color, compare_pass(dec, acc, dec_o, acc_o, band_o,
                                                          wsum=exchange_weight_sum(spec)))


def test_band_wait_timeout_is_reported(P):
    """The test hook makes every band wait for bytes no copy delivers: each wait
    gives up after its bound, no band is updated, mmc_observables reports
    MMC_ERR_TIMEOUT once, and the GPU keeps working (a normal context runs and
    agrees with the per-block pass)."""
    spec = W.chiral(128, 300.0)
    m4 = W.random_state(128 * 128, 5, 0.4, 0.6)
    g = P.MMC(spec, demag=1, sweep_tiles=1, wait_test=1, wait_polls=2000, adapt=0)
    g.set_m(m4)
    g.sweep(2, 1)
    with pytest.raises(P.MmcError) as ei:
        g.observables(0)
    assert ei.value.status == -3
    assert np.array_equal(g.get_m(0), m4)          # no band was updated
    g.observables(0)                               # the error word was cleared
    a = P.MMC(spec, demag=1, sweep_tiles=1)
    a.set_m(m4)
    a.sweep(100, 4)
    ob = a.observables(0)
    assert ob["nonfinite"] == 0 and 0.2 < ob["acc_rate"] < 0.8
