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


def _oracle_loop(spec, fields, chain, seed, chunk, threshold, min_chunks, max_chunks, every):
    """The Sec. III loop protocol on one oracle chain (runs in a spawned
    process): per field, chunks of `chunk` iterations averaging a snapshot every
    `every` iterations, until at least min_chunks chunks ran and the last two
    chunk averages of m along the field differ by less than threshold.  Returns
    the accepted chunk average per field and the chunks used."""
    import numpy as np
    import oracle as O
    o = O.Oracle(spec)
    me = O.me(float(spec["T"]), float(spec["Tc"]))
    m = np.zeros((o.n, 3))
    m[:, 0] = me
    st = O.new_state(seed=seed, chain=chain, theta_deg=30.0, adapt=True, demag_mode=1)
    mpar, used = [], []
    for B in fields:
        B = np.asarray(B, dtype=np.float64)
        bhat = B / np.linalg.norm(B) if np.linalg.norm(B) > 0 else np.array([1.0, 0.0, 0.0])
        o.set_field(B)
        hist = []
        while len(hist) < max_chunks:
            m, _, ob = o.run(m, chunk, st, obs_every=every)
            hist.append(float(np.dot(ob["mean_m"], bhat)))
            if len(hist) >= min_chunks and abs(hist[-1] - hist[-2]) < threshold:
                break
        mpar.append(hist[-1])
        used.append(len(hist))
    return mpar, used


@pytest.mark.gpu
def test_gpu_loop_matches_oracle_within_3_se():
    """The field loop of Sec. III (2000-iteration chunks, at least two, accepted
    when consecutive chunk averages of m along the field differ by < 0.01) on a
    16 x 16 film of 4 nm cells with demag, fields +100, +40, 0, -40, -100 mT
    along x: 32 GPU chains (one batch, the library's hysteresis driver) against
    16 oracle chains (other seeds) running the same protocol; at every field the
    chain means of the accepted m along the field agree within 3 standard
    errors."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    from gpu_common import lib_or_skip, welch_z
    P = lib_or_skip()
    import oracle as O
    import workloads as W
    spec = W.film256(16, B_mT=0.0)
    fields = [(b * 1e-3, 0.0, 0.0) for b in (100.0, 40.0, 0.0, -40.0, -100.0)]
    ng, no = 32, 16
    args = dict(chunk=2000, threshold=0.01, min_chunks=2, max_chunks=12, every=10)
    with cf.ProcessPoolExecutor(max_workers=max(1, min(no, (os.cpu_count() or 2) - 1)),
                                mp_context=mp.get_context("spawn")) as ex:
        fut = [ex.submit(_oracle_loop, spec, fields, c, 500 + c, **args) for c in range(no)]
        me = O.me(300.0, 870.0)
        g = P.MMC([spec] * ng, demag=1, fft_variant=1)
        for k in range(ng):
            g.set_m(W.uniform_state(16 * 16, (1, 0, 0), me), k)
        out = hysteresis(g, fields, seed=7, chunk=args["chunk"], threshold=args["threshold"],
                         min_chunks=args["min_chunks"], max_chunks=args["max_chunks"],
                         sample_every=args["every"])
        res = [f.result() for f in fut]
    gm = np.array(out["m_par"])                      # [field, chain]
    om = np.array([r[0] for r in res]).T             # [field, chain]
    for f in range(len(fields)):
        z = welch_z(gm[f], om[f])
        print("field %+6.1f mT: gpu %.5f oracle %.5f z %+.2f chunks gpu %.2f oracle %.2f"
              % (fields[f][0] * 1e3, gm[f].mean(), om[f].mean(), z, np.mean(out["chunks"][f]),
                 np.mean([r[1][f] for r in res])))
        assert abs(z) < 3.0, (f, z)
