"""GPU tests of whole runs: determinism (graphs vs eager, checkpoint/resume
bitwise), cone adaptation (Sec. II) and equilibrium observables of the
permalloy 32x32 film against the oracle within 3 standard errors."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def test_graph_and_eager_runs_are_identical(P):
    spec = W.chiral(64, 300.0)
    a = P.MMC(spec, demag=1, use_graphs=1)
    b = P.MMC(spec, demag=1, use_graphs=0)
    for g in (a, b):
        g.init_random(4)
        g.sweep(37, 9)
        g.sweep(250, 9)
    assert np.array_equal(a.get_m(), b.get_m())
    assert a.observables()["theta_deg"] == b.observables()["theta_deg"]


def test_checkpoint_resume_bitwise(P):
    spec = W.film256(64, B_mT=10.0)
    a = P.MMC(spec, demag=1)
    a.sweep(170, 3)
    ref = P.MMC(spec, demag=1)
    ref.sweep(70, 3)
    blob = ref.checkpoint()
    b = P.MMC(spec, demag=1)
    b.restore(blob)
    b.sweep(100, 3)
    assert np.array_equal(a.get_m(), b.get_m())


def test_cone_adaptation_follows_rule(P):
    spec = W.permalloy32()
    g = P.MMC(spec, theta0_deg=30.0)
    thetas = []
    for _ in range(5):
        g.sweep(100, 1)
        ob = g.observables()
        thetas.append(ob["theta_deg"])
        exp = O.adapt_theta(thetas[-2] if len(thetas) > 1 else 30.0, round(ob["acc_rate"] * 1024 * 100),
                            1024 * 100)
        assert ob["theta_deg"] == exp


def blocked_se(x, nblocks=20):
    x = np.asarray(x)
    nb = len(x) // nblocks
    b = x[: nb * nblocks].reshape(nblocks, nb).mean(1)
    return b.std(ddof=1) / math.sqrt(nblocks)


def test_equilibrium_permalloy32_matches_oracle(P):
    spec = W.permalloy32()
    n = 1024
    me = O.me(300.0, 870.0)
    m0 = W.uniform_state(n, (1, 0, 0), me)
    # GPU: 10^4 sweeps with adaptation, snapshots every sweep after 2000
    g = P.MMC(spec)
    g.set_m(m0)
    g.sweep(2000, 1)
    gx, gl = [], []
    for _ in range(80):
        g.sweep_sampled(100, 1, 1)
        ob = g.observables(reset=True)
        gx.append(ob["mean_m"][0])
        gl.append(ob["mean_len"])
    # oracle: same protocol, its own Philox streams (seed 2)
    o = O.Oracle(spec)
    st = O.new_state(seed=2, theta_deg=30.0, adapt=True, demag_mode=0)
    m = m0[:, :3].astype(np.float64)
    m, _, _ = o.run(m, 2000, st)
    ox, ol = [], []
    for _ in range(80):
        m, _, obs = o.run(m, 100, st, obs_every=1)
        ox.append(obs["mean_m"][0])
        ol.append(obs["mean_len"])
    for a, b in ((gx, ox), (gl, ol)):
        se = math.hypot(blocked_se(a), blocked_se(b))
        assert abs(np.mean(a) - np.mean(b)) < 3 * se + 1e-12, (np.mean(a), np.mean(b), se)
