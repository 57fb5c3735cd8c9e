"""GPU parity of the per-term size of the trial moves (App. B, Fig. 11) against
the oracle: the same state, random numbers, cone angle and frozen field give the
same mean |dF| / kT per term (FP32 terms against FP64: 2e-4 relative per term)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def full_spec(mesh, demag=False, pbc=(False, False, False)):
    return W._base(mesh, (3e-9, 3e-9, 2e-9), pbc=pbc, A0=1.2e-11, D0=1.1e-3, K1=3e5, K2=2e4,
                   eA=(0.3, 0.2, 0.93), Tc=650.0, T=330.0, Ms0=7e5, B=(0.02, -0.01, 0.05), demag=demag)


CASES = {
    "film_demag": (full_spec((48, 40, 1), demag=True), 2e-4),
    "film3d": (full_spec((12, 10, 4), demag=True), 2e-4),
    "periodic": (full_spec((32, 32, 1), demag=True, pbc=(True, True, False)) | {"demag_images": 3}, 2e-4),
    "cubic": (full_spec((20, 16, 2)) | {"aniso": "cubic", "K1": 4.8e5, "K2": -1e5}, 2e-4),
    "granular": (W.granular_chain(40, 3), 2e-4),
}


def compare(g_terms, o_terms, rel):
    scale = np.abs(o_terms).sum()
    for k in range(6):
        assert abs(g_terms[k] - o_terms[k]) <= rel * abs(o_terms[k]) + 1e-7 * scale, (k, g_terms, o_terms)


@pytest.mark.parametrize("name", list(CASES))
def test_trial_terms_match_oracle(P, name):
    spec, rel = CASES[name]
    n = int(np.prod(spec["mesh"]))
    m4 = W.random_state(n, 13, 0.6, 0.95)
    g = P.MMC(spec, demag=int(bool(spec.get("demag"))))
    g.set_m(m4)
    o = O.Oracle(spec)
    for sweep, theta in ((0, 30.0), (4711, 8.0)):
        gt = g.trial_terms(0, sweep, 21, theta)
        ot = o.trial_terms(m4[:, :3].astype(np.float64), None, sweep, 0, 21, theta)
        print(name, sweep, theta, "gpu", np.array2string(gt, precision=6), "oracle", np.array2string(ot, precision=6))
        compare(gt, ot, rel)
    # the state is not changed
    assert np.array_equal(g.get_m(), m4)


def test_trial_terms_in_a_batch_use_the_chain_index(P):
    specs = [W.permalloy32(16), full_spec((24, 20, 1), demag=True)]
    g = P.MMC(specs, demag=1)
    m4 = W.random_state(24 * 20, 5, 0.6, 0.9)
    g.set_m(m4, 1)
    gt = g.trial_terms(1, 17, 3, 25.0)
    ot = O.Oracle(specs[1]).trial_terms(m4[:, :3].astype(np.float64), None, 17, 1, 3, 25.0)
    compare(gt, ot, 2e-4)
    # a negative angle takes the chain's current cone angle (30 degrees at create)
    assert np.array_equal(g.trial_terms(1, 17, 3, -1.0), g.trial_terms(1, 17, 3, 30.0))


def test_trial_term_averages_driver(P):
    from paper_2106_05593_gb300 import drivers
    g = P.MMC(full_spec((32, 32, 1), demag=True), demag=1)
    g.init_random(2)
    res = drivers.trial_term_averages(g, 0, 3, 20, 7)
    assert set(res) == set(drivers.TERM_NAMES)
    assert all(np.isfinite(v) and v >= 0 for v in res.values())
    assert res["exchange"] > 0 and res["demag"] > 0
