"""GPU tests of the batch-wide state and observables calls (mmc_set_m_all,
mmc_get_m_all, mmc_observables_all): one call for every chain of a batch gives
exactly what the per-chain calls give, for the current state and for sampled
snapshots, including the reset of the accumulators; a non-finite value anywhere
in the batch leaves every chain unchanged."""
import numpy as np
import pytest

import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def _batch():
    return [W.chiral(48, 300.0), W.permalloy32(), W.chiral(40, 590.0) | {"mesh": (40, 26, 1)},
            W.granular_chain(64, 2, demag=True)]


def _same_obs(a, b):
    for key in ("mean_m", "mean_len", "mean_len2", "nsnap", "nonfinite", "acc_rate", "theta_deg", "sweeps", "hist"):
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key


def test_set_and_get_all_match_per_chain_calls(P):
    specs = _batch()
    a = P.MMC(specs, demag=1)
    b = P.MMC(specs, demag=1)
    states = [W.random_state(int(np.prod(sp["mesh"])), 90 + k, 0.4, 0.9) for k, sp in enumerate(specs)]
    a.set_m_all(np.concatenate(states))
    for k, m in enumerate(states):
        b.set_m(m, k)
    allm = a.get_m_all()
    off = 0
    for k, m in enumerate(states):
        n = m.shape[0]
        assert np.array_equal(allm[off:off + n], b.get_m(k))
        assert np.array_equal(a.get_m(k), m)
        off += n
    assert off == allm.shape[0]
    # the same iterations from the same states stay identical
    for g in (a, b):
        g.sweep(120, 7)
    for k in range(len(specs)):
        assert np.array_equal(a.get_m(k), b.get_m(k))


def test_observables_all_match_per_chain_calls(P):
    specs = _batch()
    a = P.MMC(specs, demag=1)
    a.init_random(4)
    a.sweep(50, 3)
    cur = a.observables_all()
    for k in range(len(specs)):
        _same_obs(cur[k], a.observables(k))
    # sampled snapshots, then the reset of every chain's accumulators
    a.sweep_sampled(200, 5, 10)
    snap = a.observables_all(reset=True)
    assert all(o["nsnap"] == 20 for o in snap)
    b = P.MMC(specs, demag=1)
    b.init_random(4)
    b.sweep(50, 3)
    b.sweep_sampled(200, 5, 10)
    for k in range(len(specs)):
        _same_obs(snap[k], b.observables(k))
    after = a.observables_all()
    assert all(o["nsnap"] == 0 for o in after)
    for k in range(len(specs)):
        _same_obs(after[k], a.observables(k))


def test_set_all_rejects_nonfinite_and_changes_nothing(P):
    specs = _batch()
    g = P.MMC(specs, demag=1)
    g.init_random(6)
    before = g.get_m_all()
    bad = before.copy()
    bad[-3, 1] = np.nan                     # in the last chain only
    with pytest.raises(P.MmcError) as ei:
        g.set_m_all(bad)
    assert ei.value.status == -4
    assert np.array_equal(g.get_m_all(), before)
