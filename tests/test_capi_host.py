"""CPU-side parity of the library's host code against the oracle: the demag
kernel the library convolves with (Newell tensor, near-field closed forms and
far-field quadrature, and the periodic image sums with the half-period rule)
equals the oracle's kernel at every offset.  Both are FP64 host computations
written independently; no GPU is used."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _lib_or_skip():
    from paper_2106_05593_gb300 import build
    try:
        build.build()
    except RuntimeError as e:   # no CUDA toolkit on this machine
        pytest.skip(str(e))
    import paper_2106_05593_gb300 as P
    P.load()
    return P


@pytest.mark.parametrize("mesh,h,pbc,images", [
    ((24, 16, 1), (2e-9, 2e-9, 2e-9), (0, 0, 0), 0),          # open: near field and quadrature ladder
    ((40, 6, 3), (5e-9, 3e-9, 2e-9), (0, 0, 0), 0),           # non-cubic cells, 3D offsets
    ((16, 8, 1), (3e-9, 2e-9, 1.5e-9), (1, 1, 0), 3),         # periodic in the plane
    ((10, 6, 4), (2e-9, 2e-9, 2e-9), (1, 0, 1), 2),           # periodic x and z, half periods 5 and 2
    ((7, 12, 1), (4e-9, 4e-9, 4e-9), (0, 1, 0), 5),           # odd open extent, periodic y
])
def test_demag_kernel_matches_oracle(mesh, h, pbc, images):
    P = _lib_or_skip()
    spec = W._base(mesh, h, pbc=tuple(bool(v) for v in pbc), demag=True, demag_images=images)
    o = O.Oracle(spec)
    nx, ny, nz = mesh
    lib = P.demag_kernel(h, mesh, pbc, images)
    ref = np.array([[[o.kernel(x, y, z) for x in range(nx)] for y in range(ny)] for z in range(nz)])
    scale = np.abs(ref).max()
    err = np.abs(lib - ref).max() / scale
    assert err < 1e-11, err


def test_demag_kernel_rejects_bad_arguments():
    P = _lib_or_skip()
    for args in (dict(images=65), dict(images=-1), dict(offsets=(0, 4, 1))):
        kw = dict(h=(2e-9,) * 3, n=(8, 8, 1), periodic=(1, 1, 0), images=2)
        kw.update(args)
        with pytest.raises(P.MmcError):
            P.demag_kernel(**kw)


@pytest.mark.parametrize("Tc", [870.0, 600.0])
def test_thermo_tables_match_oracle(Tc):
    """m_e, chi, sigma and the Eq. 7 free-energy differences, library host code
    against the oracle, across temperatures below, near, at and above Tc."""
    P = _lib_or_skip()
    V, Ms0 = (4e-9) ** 3, 8e5
    Ts = np.array([20.0, 300.0, 0.9 * Tc, Tc - 0.5, Tc - 1e-4, Tc + 1e-4, Tc + 3.0, 1.5 * Tc])
    t = P.thermo(Ts, Tc, V, Ms0, sigma_cap=0.03)
    for k, T in enumerate(Ts):
        # within 1 mK of Tc both sides evaluate 1 mK away; the tables are
        # conditioned like 1 / |1 - T/Tc| there
        Te = T if abs(T - Tc) >= 1e-3 else Tc + (1e-3 if T > Tc else -1e-3)
        rel = 1e-12 + 1e-15 / abs(1.0 - Te / Tc)
        assert t["me"][k] == pytest.approx(O.me(T, Tc), rel=rel, abs=1e-300), (T, "me")
        assert t["chi"][k] == pytest.approx(O.chi(T, Tc), rel=rel), (T, "chi")
        assert t["sigma"][k] == pytest.approx(O.sigma(T, Tc, V, Ms0, cap=0.03), rel=rel), (T, "sigma")
        for m1, m2 in ((0.3, 0.9), (0.05, 0.5), (0.7, 1.1)):
            want = O.long_energy(m1, T, Tc, V, Ms0) - O.long_energy(m2, T, Tc, V, Ms0)
            got = t["c2"][k] * (m1 ** 2 - m2 ** 2) + t["c4"][k] * (m1 ** 4 - m2 ** 4)
            scale = abs(O.long_energy(m1, T, Tc, V, Ms0)) + abs(O.long_energy(m2, T, Tc, V, Ms0))
            assert abs(got - want) <= (1e-11 + 1e-15 / abs(1.0 - Te / Tc)) * scale + 1e-300, (T, m1, m2, got, want)
    with pytest.raises(P.MmcError):
        P.thermo([300.0, -1.0], Tc, V, Ms0)
