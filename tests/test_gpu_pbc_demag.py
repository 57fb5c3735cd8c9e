"""GPU parity of the periodic demag convolution (films periodic in the plane,
Sec. III-IV) against the oracle's truncated image sum, through the C ABI.

- FP64 field: 1e-9 relative on 2D (interleaved kernels) and 3D (generic
  kernels) meshes, periodic along x, y, both, or all three axes; periodic
  extents that are powers of two (>= 8) take the circular transforms, the
  others the zero-padded ones with the periodized kernel.
- The GPU field of a cosine mode equals the thin-film closed form.
- Sublattice passes and whole iterations with the FP32 / FP64 / cuFFT field:
  decisions within the FP32 bound of the open-boundary tests.
- A batch mixing open and periodic chains (different kernels in one launch).
- The serial form (App. B) with the periodic field, energies and the gradient.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import compare_pass, lib_or_skip, oracle_pass

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def pfilm(mesh, h, pbc, images, **kw):
    return W._base(mesh, h, pbc=pbc, demag=True, demag_images=images, Ms0=6e5, **kw)


FIELD_CASES = [
    ((48, 40, 1), (4e-9, 4e-9, 4e-9), (1, 1, 0), 4),
    ((64, 8, 1), (2e-9, 3e-9, 1e-9), (1, 0, 0), 6),
    ((10, 32, 1), (3e-9, 2e-9, 2e-9), (0, 1, 0), 5),
    ((16, 12, 4), (3e-9, 2e-9, 2.5e-9), (1, 1, 0), 3),
    ((8, 6, 4), (2e-9, 2e-9, 2e-9), (1, 1, 1), 1),
    ((128, 64, 1), (2e-9, 2e-9, 1e-9), (1, 1, 0), 6),
]


@pytest.mark.parametrize("mesh,h,pbc,images", FIELD_CASES)
def test_periodic_demag_field_fp64(P, mesh, h, pbc, images):
    n = int(np.prod(mesh))
    spec = pfilm(mesh, h, pbc, images)
    m4 = W.random_state(n, 5, 0.5, 1.0)
    g = P.MMC(spec, demag=1)
    g.set_m(m4)
    Hg = g.demag_field(0)
    Ho = O.Oracle(spec).demag_field(m4[:, :3].astype(np.float64), "direct" if n <= 4096 else "fft")
    scale = np.abs(Ho).max()
    err = np.abs(Hg - Ho).max() / scale
    print("periodic demag fp64", mesh, pbc, images, err)
    assert err < 1e-9


def test_gpu_cosine_mode_closed_form(P):
    """M_z = cos(2 pi x / L) in a film periodic in the plane: the field is
    -S M_z with S the alias sum of the charge-sheet factor (1 - e^{-qt}) / (qt)."""
    h = (2e-9, 2e-9, 2e-9)
    mesh = (32, 16, 1)
    spec = pfilm(mesh, h, (1, 1, 0), 10)
    k = 2 * np.pi / (mesh[0] * h[0])
    x = (np.arange(mesh[0]) + 0.5) * h[0]
    c = np.broadcast_to(np.cos(k * x)[None, :], (mesh[1], mesh[0])).reshape(-1)
    m4 = np.zeros((c.size, 4), dtype=np.float32)
    m4[:, 2] = c
    g = P.MMC(spec, demag=1)
    g.set_m(m4)
    Hz = g.demag_field(0)[:, 2]
    cz = m4[:, 2].astype(np.float64)
    S = -(Hz * cz).sum() / (cz * cz).sum() / spec["Ms0"]
    M = 200000
    mm = np.arange(-M, M + 1, dtype=np.float64)
    q = np.abs(k + 2 * np.pi * mm / h[0])
    u = 0.5 * k * h[0] + np.pi * mm
    exp = float(np.sum((np.sin(u) / u) ** 2 * (-np.expm1(-q * h[2]) / (q * h[2]))))
    assert abs(S - exp) < 3e-5 * exp, (S, exp)


def test_pass_with_periodic_demag(P):
    spec = pfilm((64, 64, 1), (4e-9, 4e-9, 4e-9), (True, True, False), 4, B=(0.02, 0.0, 0.0), A0=1.3e-11)
    m4 = W.smooth_state(spec["mesh"], 3, 0.86)
    o = O.Oracle(spec)
    H = o.demag_field(m4[:, :3].astype(np.float64), "fft")
    # every FP32 kernel variant, the FP64 kernels and the cuFFT comparison path
    for fp64, cufft, variant in ((0, 0, 1), (0, 0, 2), (0, 0, 3), (1, 0, 0), (0, 1, 0)):
        g = P.MMC(spec, demag=1, demag_fp64=fp64, demag_cufft=cufft, fft_variant=variant)
        for color in (0, 1):
            g.set_m(m4)
            dec_g, acc_g = g.pass_debug(0, color, 5, 3, 25.0)
            _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 5, 0, 3, 25.0, H=H, o=o)
            print("periodic film64 fp64=%d cufft=%d variant=%d" % (fp64, cufft, variant), color,
                  compare_pass(dec_g, acc_g, dec_o, acc_o, band_o))


def test_batch_of_open_and_periodic_chains(P):
    specs = [W.film256(64, B_mT=20.0),
             pfilm((64, 64, 1), (4e-9, 4e-9, 4e-9), (1, 1, 0), 4),
             pfilm((48, 32, 1), (4e-9, 4e-9, 4e-9), (1, 0, 0), 6),
             pfilm((64, 64, 1), (4e-9, 4e-9, 4e-9), (1, 1, 0), 0)]          # periodic exchange, open demag
    g = P.MMC(specs, demag=1)
    for k, sp in enumerate(specs):
        n = int(np.prod(sp["mesh"]))
        m4 = W.random_state(n, 60 + k, 0.5, 1.0)
        g.set_m(m4, k)
        Hg = g.demag_field(k)
        o = O.Oracle(sp)
        Ho = o.demag_field(m4[:, :3].astype(np.float64), "fft")
        err = np.abs(Hg - Ho).max() / np.abs(Ho).max()
        print("batch chain", k, sp["mesh"], sp.get("demag_images", 0), err)
        assert err < 1e-9
        for color in (0, 1):
            g.set_m(m4, k)
            dec_g, acc_g = g.pass_debug(k, color, 9, 5, 30.0)
            _, acc_o, dec_o, band_o = oracle_pass(sp, m4, color, 9, k, 5, 30.0, H=Ho, o=o)
            compare_pass(dec_g, acc_g, dec_o, acc_o, band_o)


def test_full_iterations_periodic_film(P):
    spec = W.chiral_periodic(64, 300.0, 4)
    n = 64 * 64
    m4 = W.smooth_state(spec["mesh"], 5, 0.86)
    g = P.MMC(spec, demag=1, adapt=0, theta0_deg=25.0)
    g.set_m(m4)
    g.sweep(3, 13)
    mg = g.get_m()[:, :3].astype(np.float64)
    st = O.new_state(seed=13, chain=0, theta_deg=25.0, adapt=False, demag_mode=1)
    mo, _, _ = O.Oracle(spec).run(m4[:, :3].astype(np.float64), 3, st)
    d = np.abs(mg - mo).max(axis=1)
    differ = int((d > 1e-5).sum())
    print("periodic full iterations: max |dm| over agreeing cells %.2e, differing cells %d"
          % (d[d <= 1e-5].max(), differ))
    assert differ <= 2


@pytest.mark.parametrize("self_term", [0, 1])
def test_serial_form_periodic(P, self_term):
    spec = pfilm((24, 16, 1), (4e-9, 4e-9, 4e-9), (1, 1, 0), 4, A0=1e-11, D0=1e-3, K1=2e5,
                 Tc=600.0, T=300.0, B=(0.02, 0.0, 0.01))
    n = 24 * 16
    m4 = W.smooth_state(spec["mesh"], 3, 0.8)
    g = P.MMC(spec, demag=1, adapt=0, theta0_deg=20.0, demag_self=self_term)
    g.set_m(m4)
    g.sweep_serial(2, 21)
    mg = g.get_m()[:, :3].astype(np.float64)
    st = O.new_state(seed=21, chain=0, theta_deg=20.0, adapt=False, demag_mode=3)
    mo, _, _ = O.Oracle(spec, demag_self=bool(self_term)).run(m4[:, :3].astype(np.float64), 2, st)
    d = np.abs(mg - mo).max(axis=1)
    moved = int((np.abs(mo - m4[:, :3]).max(axis=1) > 0).sum())
    differ = int((d > 1e-5).sum())
    print("serial periodic self=%d: moved %d, differing %d" % (self_term, moved, differ))
    assert moved > n // 4
    assert differ <= 3


def test_energy_and_gradient_periodic(P):
    import torch
    spec = pfilm((32, 20, 2), (4e-9, 4e-9, 4e-9), (1, 1, 0), 3, A0=1e-11, D0=1.5e-3, K1=8e5,
                 Tc=600.0, T=300.0, B=(0.01, -0.02, 0.03))
    n = int(np.prod(spec["mesh"]))
    me = O.me(spec["T"], spec["Tc"])
    m = W.random_state(n, 3, 0.8 * me, me)[:, :3].astype(np.float64)
    g = P.MMC(spec, demag=1)
    o = O.Oracle(spec)
    go, _, Eo = o.energy_grad(m)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda").contiguous()
    E, dEdm, _ = g.energy_grad(mt)
    d = dEdm.cpu().numpy()
    assert np.linalg.norm(d - go) / np.linalg.norm(go) < 1e-6
    assert np.abs(np.asarray(E) - Eo).max() < 1e-9 * np.abs(Eo[1:]).sum()
    m4 = np.zeros((n, 4), dtype=np.float32)
    m4[:, :3] = m
    g.set_m(m4)
    Eg = g.energy(0)
    Ee = o.energy(m4[:, :3].astype(np.float64))
    for k in range(7):
        assert Eg[k] == pytest.approx(Ee[k], abs=1e-9 * np.abs(Ee[1:]).sum()), (k, Eg, Ee)


def test_images_argument_is_validated(P):
    for bad in (-1, 65):
        with pytest.raises(P.MmcError):
            P.MMC(pfilm((16, 16, 1), (2e-9, 2e-9, 2e-9), (1, 1, 0), bad), demag=1)
    # images without a periodic axis leave the convolution open
    spec = pfilm((16, 12, 1), (2e-9, 2e-9, 2e-9), (0, 0, 0), 5)
    m4 = W.random_state(16 * 12, 2, 0.5, 1.0)
    g = P.MMC(spec, demag=1)
    g.set_m(m4)
    Ho = O.Oracle(spec | {"demag_images": 0}).demag_field(m4[:, :3].astype(np.float64))
    assert np.abs(g.demag_field(0) - Ho).max() < 1e-9 * np.abs(Ho).max()


def test_granular_periodic_chain(P):
    """Per-cell Ms0 (grains) with the periodic field, circular transforms."""
    spec = W.granular_chain(32, 6) | {"pbc": (True, True, False), "demag_images": 3}
    n = 32 * 32
    m4 = W.random_state(n, 17, 0.6, 0.9)
    g = P.MMC(spec, demag=1)
    g.set_m(m4)
    o = O.Oracle(spec)
    Ho = o.demag_field(m4[:, :3].astype(np.float64), "direct")
    # per-cell Ms0 is stored in FP32 on the device (relative rounding 2^-24 per source)
    assert np.abs(g.demag_field(0) - Ho).max() < 1e-7 * np.abs(Ho).max()
    for color in (0, 1):
        g.set_m(m4)
        dec_g, acc_g = g.pass_debug(0, color, 3, 9, 30.0)
        _, acc_o, dec_o, band_o = oracle_pass(spec, m4, color, 3, 0, 9, 30.0, H=Ho, o=o)
        compare_pass(dec_g, acc_g, dec_o, acc_o, band_o)


def test_minimizer_with_periodic_demag(P):
    """SDesc (Sec. III) on a film periodic in the plane: same minimum as the
    oracle's minimizer with the periodic kernel."""
    s = pfilm((16, 8, 1), (3e-9, 3e-9, 2e-9), (1, 1, 0), 2, A0=1.2e-11, D0=1e-3, K1=3e5, Tc=650.0,
              T=300.0, B=(0.02, 0.01, 0.05))
    m4 = W.smooth_state(s["mesh"], 3, 0.8)
    g = P.MMC(s, demag=1)
    g.set_m(m4)
    r = g.minimize(0, maxit=20000, tol=1e-7)
    assert r["converged"], r
    o = O.Oracle(s)
    mo, ok, it, tq = o.sdesc(m4[:, :3].astype(np.float64), maxit=20000, tol=1e-7)
    assert ok
    mg = g.get_m()[:, :3].astype(np.float64)
    assert np.abs(mg - mo).max() < 2e-5
    assert r["energy"][0] == pytest.approx(o.energy(mo)[0], rel=1e-9)

