"""GPU tests of the differentiable energy (forward + hand-written backward)
against the oracle's analytic gradient, central finite differences and
torch.autograd.gradcheck; FP64 to 1e-6 and FP32 to 1e-4 (norm-wise relative)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def state(spec, seed):
    """|m| uniform in [0.8, 1.0] m_e, random directions (differentiable-energy workload)."""
    n = int(np.prod(spec["mesh"]))
    me = O.me(spec["T"], spec["Tc"])
    return W.random_state(n, seed, 0.8 * me, 1.0 * me)[:, :3].astype(np.float64)


@pytest.mark.parametrize("mesh", [(16, 12, 4), (24, 20, 1)])
def test_gradient_matches_oracle(P, mesh):
    import torch
    spec = W.energy3d(mesh[0], mesh[2])
    spec["mesh"] = mesh
    spec["B"] = (0.01, -0.02, 0.03)
    m = state(spec, 3)
    g = P.MMC(spec, demag=1)
    o = O.Oracle(spec)
    go, dpo, Eo = o.energy_grad(m)
    for dt, tol in ((torch.float64, 1e-6), (torch.float32, 1e-4)):
        mt = torch.tensor(m, dtype=dt, device="cuda").contiguous()
        E, dEdm, dEdp = g.energy_grad(mt)
        d = dEdm.double().cpu().numpy()
        rel = np.linalg.norm(d - go) / np.linalg.norm(go)
        assert rel < tol, (dt, rel)
        floor = 1e-3 * np.sqrt((go ** 2).mean())
        assert (np.abs(d - go) / (np.abs(go) + floor)).max() < 100 * tol
        scale = np.abs(Eo[1:]).sum()
        assert np.abs(E - Eo).max() < (1e-9 if dt == torch.float64 else 1e-6) * scale
        # parameter gradients: closed forms of the oracle (uniform material)
        tb = o.tables()
        assert dEdp[0] == pytest.approx(dpo[0], rel=tol)
        assert dEdp[1] == pytest.approx(dpo[1], rel=tol)
        assert dEdp[2] == pytest.approx(dpo[2], rel=tol)
        assert dEdp[3] == pytest.approx(dpo[3], rel=tol)
        assert dEdp[4] == pytest.approx(-Eo[5] / tb["chi"][0], rel=tol)


def test_gradient_central_differences(P):
    import torch
    spec = W.energy3d(8, 4)
    spec["mesh"] = (8, 6, 4)
    m = state(spec, 5)
    g = P.MMC(spec, demag=1)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda").contiguous()
    _, dEdm, dEdp = g.energy_grad(mt)
    d = dEdm.cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(1)
    for _ in range(12):
        i = int(rng.integers(0, m.shape[0]))
        a = int(rng.integers(0, 3))
        mp = mt.clone(); mp[i, a] += h
        mm = mt.clone(); mm[i, a] -= h
        fd = (g.energy_grad(mp, grad=False)[0][0] - g.energy_grad(mm, grad=False)[0][0]) / (2 * h)
        assert d[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(d).max())
    base = np.array([6e5, 1e-11, 1.5e-3, 8e5, O.chi(300.0, 600.0)])
    for k in range(5):
        dp = base.copy(); dp[k] *= 1 + 1e-6
        dm_ = base.copy(); dm_[k] *= 1 - 1e-6
        fd = (g.energy_grad(mt, dp, grad=False)[0][0] - g.energy_grad(mt, dm_, grad=False)[0][0]) / (2e-6 * base[k])
        assert dEdp[k] == pytest.approx(fd, rel=1e-6), k


def test_autograd_function_gradcheck(P):
    import torch
    from paper_2106_05593_gb300.energy import Energy
    spec = W.energy3d(4, 2)
    spec["mesh"] = (4, 4, 2)
    g = P.MMC(spec, demag=1)
    m = torch.tensor(state(spec, 7), dtype=torch.float64, device="cuda", requires_grad=True)
    # scaled parameters keep gradcheck's absolute tolerances meaningful
    params = torch.tensor([6e5, 1e-11, 1.5e-3, 8e5, O.chi(300.0, 600.0)], dtype=torch.float64,
                          requires_grad=True)
    E = Energy.apply(m, params, g, 0)
    E.backward()
    _, dEdm, dEdp = g.energy_grad(m.detach())
    assert torch.allclose(m.grad, dEdm, rtol=1e-12, atol=0)
    assert np.allclose(params.grad.numpy(), dEdp, rtol=1e-12, atol=0)
    scale = float(E.abs()) + 1e-30
    f = lambda mm: Energy.apply(mm, params.detach(), g, 0) / scale
    assert torch.autograd.gradcheck(f, (m,), eps=1e-7, atol=1e-5, rtol=1e-4)


def test_full_size_energy3d_sampled(P):
    """256 x 256 x 4 (the differentiable-energy workload): FP64 gradient against
    the oracle's analytic gradient on every cell, FP32 within 1e-4."""
    import torch
    spec = W.energy3d(256, 4)
    m = state(spec, 1)
    g = P.MMC(spec, demag=1)
    go, _, Eo = O.Oracle(spec).energy_grad(m)
    for dt, tol in ((torch.float64, 1e-6), (torch.float32, 1e-4)):
        mt = torch.tensor(m, dtype=dt, device="cuda").contiguous()
        E, dEdm, _ = g.energy_grad(mt)
        d = dEdm.double().cpu().numpy()
        rel = np.linalg.norm(d - go) / np.linalg.norm(go)
        print("energy3d 256x256x4", dt, "grad rel", rel, "E rel", abs(E[0] - Eo[0]) / abs(Eo[0]))
        assert rel < tol
        # time one forward + backward evaluation (the call returns after the
        # device work and the read-back of the energies), after a warm-up
        import time
        for _ in range(3):
            g.energy_grad(mt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            g.energy_grad(mt)
        torch.cuda.synchronize()
        print("energy3d 256x256x4", dt, "forward+backward ms %.3f" % ((time.perf_counter() - t0) * 100))
