"""GPU tests of the serial form of the method (App. B) against the oracle's
serial sweep (cells in index order, demag field updated after every accepted
move, Eq. 14 against the current field, optionally with the self term)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def _case(name):
    if name == "film":                      # 2D, DMI, anisotropy, field, demag
        spec = W._base((32, 24, 1), (4e-9, 4e-9, 4e-9), Ms0=6e5, A0=1e-11, D0=1.5e-3, K1=3e5,
                       Tc=600.0, T=300.0, B=(0.02, 0.0, 0.01), demag=True)
        m4 = W.smooth_state(spec["mesh"], 3, 0.8)
    elif name == "film3d":                  # six tensor components
        spec = W._base((10, 8, 3), (3e-9, 3e-9, 3e-9), B=(0.0, 0.03, 0.0), demag=True, T=500.0)
        m4 = W.smooth_state(spec["mesh"], 4, 0.75)
    elif name == "granular":                # per-cell tables, grains, hotspot
        spec = W.granular_chain(40, 5)
        m4 = W.smooth_state(spec["mesh"], 6, 0.7)
    elif name == "nodemag":                 # serial index-order Metropolis sweep
        spec = W.permalloy32(24)
        m4 = W.random_state(24 * 24, 7, 0.8, 0.9)
    elif name == "global":                  # too large for shared memory: global-memory walk
        spec = W._base((72, 64, 1), (4e-9, 4e-9, 4e-9), B=(0.01, 0.0, 0.0), demag=True)
        m4 = W.smooth_state(spec["mesh"], 8, 0.86)
    else:
        raise ValueError(name)
    return spec, m4


@pytest.mark.parametrize("name,self_term", [("film", 0), ("film", 1), ("film3d", 0), ("film3d", 1),
                                            ("granular", 0), ("nodemag", 0), ("global", 0), ("global", 1)])
def test_serial_sweeps_match_oracle(P, name, self_term):
    """Two serial iterations from the same state, seed and cone (Eq. 14 against
    the current field, with or without the self term): every cell ends equal to
    FP32 rounding unless a decision sits inside the FP32 bound (a flip then
    changes that cell, and through the field and its neighbours maybe a few
    more later in the walk)."""
    spec, m4 = _case(name)
    n = int(np.prod(spec["mesh"]))
    g = P.MMC(spec, demag=int(bool(spec.get("demag"))), adapt=0, theta0_deg=20.0, demag_self=self_term)
    g.set_m(m4)
    g.sweep_serial(2, 21)
    mg = g.get_m()[:, :3].astype(np.float64)
    o = O.Oracle(spec, demag_self=bool(self_term))
    st = O.new_state(seed=21, chain=0, theta_deg=20.0, adapt=False, demag_mode=3)
    mo, _, _ = o.run(m4[:, :3].astype(np.float64), 2, st)
    d = np.abs(mg - mo).max(axis=1)
    moved = int((np.abs(mo - m4[:, :3]).max(axis=1) > 0).sum())
    differ = int((d > 1e-5).sum())
    print("serial %s self=%d: %d cells, %d moved, max |dm| over agreeing cells %.2e, differing %d"
          % (name, self_term, n, moved, d[d <= 1e-5].max(), differ))
    assert moved > n // 4
    assert differ <= 3


def test_serial_continues_the_sweep_counter(P):
    """Two calls of one iteration equal one call of two (bitwise), and the
    serial and parallel forms share the counter: a parallel iteration after a
    serial one uses sweep index 1."""
    spec, m4 = _case("film")
    a = P.MMC(spec, demag=1, adapt=0)
    b = P.MMC(spec, demag=1, adapt=0)
    a.set_m(m4)
    b.set_m(m4)
    a.sweep_serial(1, 5)
    a.sweep_serial(1, 5)
    b.sweep_serial(2, 5)
    assert np.array_equal(a.get_m(), b.get_m())
    a.sweep(1, 5)
    c = P.MMC(spec, demag=1, adapt=0)
    c.set_m(b.get_m())
    c.sweep_serial(2, 99)             # advance the counter by two with other numbers
    c.set_m(b.get_m())
    c.sweep(1, 5)
    assert np.array_equal(a.get_m(), c.get_m())


def test_serial_batch_of_chains(P):
    """A batch runs every chain's walk in its own block.  Uniform batch: chain 0
    equals the same chain run alone, bit for bit.  Mixed batch (a per-cell
    granular chain makes every chain of the batch use per-cell tables): every
    chain agrees with the oracle's serial walk under its own chain index."""
    names = ["film", "film3d", "granular"]
    specs = [_case(nm)[0] for nm in names]
    states = [_case(nm)[1] for nm in names]
    u = P.MMC(specs[:2], demag=1, adapt=0)
    for k in range(2):
        u.set_m(states[k], k)
    u.sweep_serial(2, 3)
    one = P.MMC([specs[0]], demag=1, adapt=0)
    one.set_m(states[0])
    one.sweep_serial(2, 3)
    assert np.array_equal(one.get_m(), u.get_m(0))
    g = P.MMC(specs, demag=1, adapt=0)
    for k, m4 in enumerate(states):
        g.set_m(m4, k)
    g.sweep_serial(2, 3)
    for k, (sp, m4) in enumerate(zip(specs, states)):
        mo, _, _ = O.Oracle(sp).run(m4[:, :3].astype(np.float64), 2,
                                   O.new_state(seed=3, chain=k, theta_deg=30.0, adapt=False, demag_mode=3))
        differ = int((np.abs(g.get_m(k)[:, :3] - mo).max(axis=1) > 1e-5).sum())
        assert differ <= 3


def test_parallel_and_serial_switching_statistics_agree(P):
    """App. B: switching of a small Permalloy element from the -x remanent state
    under a +x field near its switching field, once with the field updated once
    per iteration (parallel form, Eq. 14 frozen field) and once after every
    accepted move (serial form).  The crossing-time distributions of 128
    chains must agree: two-sample Kolmogorov-Smirnov distance below the 0.1%
    critical value 1.95 sqrt(2/128) = 0.244, medians within 10%."""
    from paper_2106_05593_gb300.drivers import switching_trace, crossing_probability
    nch, mesh = 128, (40, 20, 1)
    spec = W._base(mesh, (5e-9, 5e-9, 5e-9), B=(0.055, 0.0, 0.0), demag=True)
    me = O.me(300.0, 870.0)
    n = int(np.prod(mesh))
    out = {}
    for serial in (False, True):
        g = P.MMC([spec] * nch, demag=1)
        for k in range(nch):
            g.set_m(W.uniform_state(n, (-1.0, 0.0, 0.0), me), k)
        its, tr = switching_trace(g, 4000, 1, every=20, serial=serial)
        crossed = np.maximum.accumulate(tr > 0, axis=0)
        first = np.where(crossed.any(axis=0), its[np.argmax(crossed, axis=0)], np.inf)
        out[serial] = (crossing_probability(tr), first)
    (pp, fp), (ps, fs) = out[False], out[True]
    ks = np.abs(pp - ps).max()
    med_p, med_s = np.median(fp), np.median(fs)
    print("App. B switching: median crossing parallel %.0f serial %.0f, KS %.3f, P(4000) %.3f %.3f"
          % (med_p, med_s, ks, pp[-1], ps[-1]))
    assert pp[-1] > 0.95 and ps[-1] > 0.95
    assert ks < 0.244
    assert abs(med_s - med_p) < 0.1 * med_p
