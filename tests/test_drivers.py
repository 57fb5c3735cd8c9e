"""Host logic of the hysteresis driver (Sec. III chunk rule), on a scripted fake
engine (no GPU), and one small GPU loop."""
import numpy as np
import pytest

from paper_2106_05593_gb300.drivers import chunk_converged, hysteresis


class FakeEngine:
    """Returns scripted chunk averages of m_x per chain."""

    def __init__(self, scripts):
        self.scripts = scripts
        self.nchains = len(scripts)
        self.pos = [0] * self.nchains
        self.calls = []

    def set_field(self, B, chain):
        self.calls.append(("field", tuple(B)))
        self.pos = [0] * self.nchains

    def sweep_sampled(self, n, seed, every):
        self.calls.append(("sweep", n))
        self.pos = [p + 1 for p in self.pos]

    def observables(self, k, reset=False):
        p = self.pos[k]
        v = self.scripts[k][min(p, len(self.scripts[k])) - 1] if p > 0 else 0.0
        return {"mean_m": np.array([v, 0.0, 0.0])}


def test_chunk_rule():
    assert not chunk_converged([0.5], 0.01)
    assert chunk_converged([0.5, 0.505], 0.01)
    assert not chunk_converged([0.5, 0.52], 0.01)
    assert chunk_converged([0.5, 0.52, 0.515], 0.01)


def test_hysteresis_spends_chunks_until_consecutive_averages_agree():
    eng = FakeEngine([[0.9, 0.895, 0.894, 0.1], [0.2, 0.5, 0.7, 0.705]])
    out = hysteresis(eng, [(0.1, 0.0, 0.0)], seed=1, chunk=2000)
    assert out["chunks"] == [[2, 4]]                  # chain 0 stops at 2, chain 1 needs 4
    assert out["m_par"][0][0] == pytest.approx(0.895)
    assert out["m_par"][0][1] == pytest.approx(0.705)
    assert out["iterations"] == 4 * 2000
    assert eng.calls[0] == ("field", (0.1, 0.0, 0.0))


def test_projection_on_the_field_direction():
    eng = FakeEngine([[0.8, 0.8]])
    out = hysteresis(eng, [(-0.05, 0.0, 0.0)], seed=1)
    assert out["m_par"][0][0] == pytest.approx(-0.8)


@pytest.mark.gpu
def test_small_gpu_loop_saturates_along_the_field():
    from gpu_common import lib_or_skip
    P = lib_or_skip()
    import workloads as W
    spec = W.film256(32, B_mT=0.0)
    g = P.MMC(spec, demag=1)
    fields = [(b * 1e-3, 0.0, 0.0) for b in (200.0, 0.0, -200.0)]
    out = hysteresis(g, fields, seed=3, chunk=200, sample_every=5)
    mp = np.array(out["m_par"])[:, 0]
    assert mp[0] > 0.8 and mp[2] > 0.8           # saturated along +x, then along -x
    assert all(c >= 2 for row in out["chunks"] for c in row)


def test_crossing_probability_is_cumulative():
    from paper_2106_05593_gb300.drivers import crossing_probability
    tr = np.array([[-1.0, -1.0, -0.5],
                   [0.2, -1.0, -0.4],
                   [-0.1, -0.9, 0.3],     # chain 0 back below: stays counted
                   [-0.3, 0.5, 0.4]])
    assert np.allclose(crossing_probability(tr), [0.0, 1 / 3, 2 / 3, 1.0])


class _FakeSerial:
    """Host-side stand-in for an MMC context: mean m_x rises by 0.1 per iteration."""
    nchains = 2

    def __init__(self):
        self.it = 0
        self.calls = []

    def sweep(self, n, seed):
        self.calls.append(("parallel", n))
        self.it += n

    def sweep_serial(self, n, seed):
        self.calls.append(("serial", n))
        self.it += n

    def observables(self, chain, reset=False):
        return {"mean_m": np.array([-1.0 + 0.1 * self.it * (chain + 1), 0.0, 0.0])}


def test_switching_trace_sequences_calls():
    from paper_2106_05593_gb300.drivers import switching_trace
    e = _FakeSerial()
    its, tr = switching_trace(e, 25, 1, every=10, serial=True)
    assert list(its) == [10, 20, 25]
    assert e.calls == [("serial", 10), ("serial", 10), ("serial", 5)]
    assert np.allclose(tr[:, 0], [0.0, 1.0, 1.5]) and np.allclose(tr[:, 1], [1.0, 3.0, 4.0])


class _FakeAngles:
    nchains = 1

    def __init__(self):
        self.calls = 0

    def sweep(self, n, seed):
        self.calls += 1

    def angle_hist(self, chain, bins, lo, hi):
        h = np.zeros(bins + 1, dtype=np.int64)
        h[0] = 3
        h[bins - 1] = 1
        h[bins] = 5                      # out of range: not part of the density
        return h, np.array([0.0, 0.0, 1.0])


def test_angular_histogram_averages_to_a_density():
    from paper_2106_05593_gb300.drivers import angular_histogram
    e = _FakeAngles()
    c, dens = angular_histogram(e, 0, 4, 10, 1, bins=10, lo=0.0, hi=1.0)
    assert e.calls == 4
    assert np.allclose(c, (np.arange(10) + 0.5) / 10)
    assert np.isclose(dens.sum() * 0.1, 1.0) and np.isclose(dens[0], 0.75 / 0.1)
