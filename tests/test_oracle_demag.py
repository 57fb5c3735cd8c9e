"""Oracle demag pins (CPU only): Newell tensor and the Eq. 14 convolution.

- Self term: trace 1 for any cuboid, 1/3 each for a cube.
- Near-field Newell formulas and the far-field cell-pair quadrature agree where
  both are accurate.
- Uniformly magnetized prisms: the discrete tensor sums equal the closed-form
  demagnetizing factors of a rectangular prism (A. Aharoni, J. Appl. Phys. 83,
  3432 (1998)) -- cube, a non-cubic prism with non-cubic cells, and the
  1024 nm x 1024 nm x 4 nm film of 256 x 256 cells of 4 nm (to 1e-6).
- FFT convolution (zero padded) equals the direct sum.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def aharoni_dz(a, b, c):
    """Demagnetizing factor along z of a prism 2a x 2b x 2c (Aharoni 1998)."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    s = ((b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
         + b / (2 * c) * math.log((ab + a) / (ab - a))
         + a / (2 * c) * math.log((ab + b) / (ab - b))
         + c / (2 * a) * math.log((bc - b) / (bc + b))
         + c / (2 * b) * math.log((ac - a) / (ac + a))
         + 2 * math.atan(a * b / (c * r))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return s / math.pi


def aharoni(Lx, Ly, Lz):
    a, b, c = Lx / 2, Ly / 2, Lz / 2
    return aharoni_dz(b, c, a), aharoni_dz(c, a, b), aharoni_dz(a, b, c)


def test_aharoni_formula_sanity():
    assert aharoni(1, 1, 1) == pytest.approx((1 / 3,) * 3, rel=1e-14)
    assert sum(aharoni(3, 7, 0.4)) == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("h", [(4e-9, 4e-9, 4e-9), (5e-9, 3e-9, 2e-9), (2e-9, 2e-9, 1e-9)])
def test_self_term_trace_and_prism(h):
    t = O.newell(h, (0, 0, 0))
    assert t[0] + t[1] + t[2] == pytest.approx(1.0, rel=1e-15)
    assert np.abs(t[3:]).max() < 1e-15
    assert tuple(t[:3]) == pytest.approx(aharoni(*h), rel=1e-12)


@pytest.mark.parametrize("h,R", [
    ((4e-9, 4e-9, 4e-9), (31, 7, 0)), ((4e-9, 4e-9, 4e-9), (20, 25, 0)),
    ((5e-9, 3e-9, 2e-9), (21, 11, 3)), ((2e-9, 2e-9, 1e-9), (15, -12, 2))])
def test_newell_and_quadrature_agree(h, R):
    # near the switch radius (20 h_max) both formulas are accurate
    X = [R[k] * h[k] for k in range(3)]
    a = O.newell(h, X)
    b = O.tensor_quad(h, X, 6)
    scale = np.abs(a[:3]).max()
    assert np.abs(a - b).max() < 1e-9 * scale


def test_tensor_symmetry():
    h = (5e-9, 3e-9, 2e-9)
    for R in [(3, 2, 1), (40, 13, 2)]:
        X = np.array([R[k] * h[k] for k in range(3)])
        t = O.tensor(h, X)
        for sx, sy, sz in [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]:
            u = O.tensor(h, X * np.array([sx, sy, sz]))
            assert u[:3] == pytest.approx(t[:3], rel=1e-13)
            assert u[3] == pytest.approx(sx * sy * t[3], rel=1e-12)
            assert u[4] == pytest.approx(sx * sz * t[4], rel=1e-12)
            assert u[5] == pytest.approx(sy * sz * t[5], rel=1e-12)


def _uniform_factor(spec, axis):
    o = O.Oracle(spec)
    m = np.zeros((o.n, 3))
    m[:, axis] = 1.0
    E = o.energy(m)[6]
    V = spec["h"][0] * spec["h"][1] * spec["h"][2]
    return E / (0.5 * O.MU0 * spec["Ms0"] ** 2 * V * o.n)


@pytest.mark.parametrize("mesh,h", [((6, 6, 6), (4e-9, 4e-9, 4e-9)),
                                    ((16, 8, 2), (5e-9, 3e-9, 2e-9))])
def test_uniform_prism_factors(mesh, h):
    s = W._base(mesh, h, demag=True, Ms0=8e5)
    L = [mesh[k] * h[k] for k in range(3)]
    ref = aharoni(*L)
    for axis in range(3):
        assert _uniform_factor(s, axis) == pytest.approx(ref[axis], abs=1e-9)


def test_thin_film_factor_256():
    s = W.film256(256)
    ref = aharoni(1024e-9, 1024e-9, 4e-9)
    Nz = _uniform_factor(s, 2)
    Nx = _uniform_factor(s, 0)
    assert Nz == pytest.approx(ref[2], abs=1e-6)
    assert Nx == pytest.approx(ref[0], abs=1e-6)


@pytest.mark.parametrize("mesh,h", [((12, 10, 1), (4e-9, 4e-9, 4e-9)),
                                    ((6, 5, 3), (5e-9, 3e-9, 2e-9))])
def test_fft_convolution_equals_direct_sum(mesh, h):
    n = mesh[0] * mesh[1] * mesh[2]
    rng = np.random.default_rng(9)
    s = W._base(mesh, h, demag=True, Ms0=rng.uniform(4e5, 9e5, n))
    o = O.Oracle(s)
    m = rng.standard_normal((n, 3))
    Hd = o.demag_field(m, "direct")
    Hf = o.demag_field(m, "fft")
    assert np.abs(Hd - Hf).max() < 1e-12 * np.abs(Hd).max()


@pytest.mark.parametrize("mesh,h", [((9, 7, 1), (4e-9, 4e-9, 4e-9)),
                                    ((5, 4, 3), (5e-9, 3e-9, 2e-9))])
def test_serial_sweep_keeps_the_field_exact(mesh, h):
    """App. B serial form: after a sweep in which the field was updated after
    every accepted move, the field equals the direct sum over the final state
    (a wrong sign, axis flip or offset direction in the update breaks this)."""
    n = mesh[0] * mesh[1] * mesh[2]
    rng = np.random.default_rng(4)
    s = W._base(mesh, h, demag=True, Ms0=rng.uniform(4e5, 9e5, n), T=600.0)
    o = O.Oracle(s)
    m = 0.8 * rng.standard_normal((n, 3)) / math.sqrt(3)
    H0 = o.demag_field(m, "direct")
    m1, H1, nacc = o.serial_sweep(m, H0, 0, 0, 17, 60.0)
    assert nacc > n // 4
    H_ref = o.demag_field(m1, "direct")
    assert np.abs(H1 - H_ref).max() < 1e-12 * np.abs(H_ref).max()

