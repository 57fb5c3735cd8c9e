"""Oracle pins for the periodic demag convolution (CPU only).

The films of Sec. III-IV are periodic in the plane; the oracle reads the
periodic Eq. 14 convolution as the lattice sum over periodic images, truncated
at ``demag_images`` images on each side, each offset taken at its minimal image
and the half-period offset split between its two minimal images.  What pins it,
independently of the oracle's own arithmetic:

- A film that is infinite in the plane, magnetized as a cosine along x (or y),
  has the thickness-averaged field of its charge sheets in closed form: for
  M_z = cos(q x) the field is -G(q) M_z and for M_x = cos(q x) it is
  -(1 - G(q)) M_x, G(q) = (1 - exp(-q t)) / (q t), while M_y = cos(q x) carries
  no charge and no field.  Cells that are uniformly magnetized and fields
  averaged over a cell (the Newell tensor's meaning) turn this into a sum over
  the aliases q = k + 2 pi m / h weighted by sinc^2(q h / 2), evaluated here
  directly.  The truncated image sum approaches it as the number of images
  grows.
- Exact covariance under circular shifts along a periodic axis (which open
  boundaries break).
- Parity at the half-period offset: odd components vanish there.
- The uniform film: H_z -> -Ms (perpendicular) and H_x -> 0 (in plane) as the
  images grow, with the finite-plate correction shrinking like 1 / (2P + 1).
"""
import numpy as np
import pytest

import oracle as O

MS = 1.0e6


def film(n, h, P, pbc=(1, 1, 0)):
    return dict(mesh=n, pbc=pbc, h=h, Ms0=MS, A0=0.0, Tc=600.0, T=300.0, demag=True,
                demag_images=P)


def alias_sum(k, h, t, kind, M=200000):
    """sum_m sinc^2(k h / 2 + pi m) g(|k + 2 pi m / h|), g = G (perpendicular
    magnetization) or 1 - G (in-plane magnetization along the modulation)."""
    m = np.arange(-M, M + 1, dtype=np.float64)
    q = np.abs(k + 2.0 * np.pi * m / h)
    u = 0.5 * k * h + np.pi * m
    s2 = (np.sin(u) / u) ** 2
    G = -np.expm1(-q * t) / (q * t)
    return float(np.sum(s2 * (G if kind == "perp" else 1.0 - G)))


def mode_response(o, n, h, axis, ell, comp):
    """-<H_comp cos(k r_axis)> / (Ms <cos^2>) for m_comp = cos(k r_axis), and the
    largest residual of H_comp from that cosine and of the other components."""
    nx, ny, nz = n
    k = 2.0 * np.pi * ell / (n[axis] * h[axis])
    r = (np.arange(n[axis]) + 0.5) * h[axis]
    c = np.cos(k * r)
    shape = [1, 1, 1]
    shape[2 - axis] = n[axis]                         # arrays are (z, y, x)
    cc = np.broadcast_to(c.reshape(shape), (nz, ny, nx))
    m = np.zeros((nz, ny, nx, 3))
    m[..., comp] = cc
    H = o.demag_field(m.reshape(-1, 3), method="fft").reshape(nz, ny, nx, 3)
    S = -(H[..., comp] * cc).sum() / (cc * cc).sum() / MS
    resid = np.abs(H[..., comp] + MS * S * cc).max() / MS
    other = max(np.abs(H[..., a]).max() for a in range(3) if a != comp) / MS
    return S, resid, other, k


@pytest.mark.parametrize("h", [(2e-9, 2e-9, 2e-9), (3e-9, 2e-9, 1.5e-9)])
@pytest.mark.parametrize("axis", [0, 1])
def test_film_cosine_modes_closed_form(h, axis):
    n = (16, 8, 1) if axis == 0 else (8, 16, 1)
    o = O.Oracle(film(n, h, 8))
    t = h[2]
    for ell in (1, 2, 5):
        # perpendicular magnetization: surface charges, -G(q)
        S, resid, other, k = mode_response(o, n, h, axis, ell, 2)
        exp = alias_sum(k, h[axis], t, "perp")
        assert abs(S - exp) < 3e-5 * exp, (ell, S, exp)
        assert resid < 1e-12 and other < 1e-12
        # in-plane along the modulation: volume charges, -(1 - G(q))
        S, resid, other, k = mode_response(o, n, h, axis, ell, axis)
        exp = alias_sum(k, h[axis], t, "inplane")
        assert abs(S - exp) < 5e-5 * exp, (ell, S, exp)
        assert resid < 1e-12
        # in-plane across the modulation: divergence free, no field
        S, resid, other, k = mode_response(o, n, h, axis, ell, 1 - axis)
        assert abs(S) < 2e-6 and other < 2e-6


def test_film_two_layers_thickness_average():
    # two cell layers: the layer-averaged field is the whole film's average
    h = (2e-9, 2e-9, 1e-9)
    n = (16, 8, 2)
    o = O.Oracle(film(n, h, 8))
    for ell in (1, 3):
        S, _, _, k = mode_response(o, n, h, 0, ell, 2)
        exp = alias_sum(k, h[0], 2 * h[2], "perp")
        assert abs(S - exp) < 3e-5 * exp


def test_image_truncation_converges():
    h = (2e-9, 2e-9, 2e-9)
    n = (16, 8, 1)
    errs = []
    for P in (1, 2, 8):
        o = O.Oracle(film(n, h, P))
        S, _, _, k = mode_response(o, n, h, 0, 1, 0)
        errs.append(abs(S - alias_sum(k, h[0], h[2], "inplane")))
    assert errs[2] < errs[1] / 10 < errs[0] / 10


@pytest.mark.parametrize("n,pbc", [((8, 6, 1), (1, 1, 0)), ((8, 4, 2), (1, 0, 0)), ((6, 8, 1), (0, 1, 0))])
def test_circular_shift_covariance(n, pbc):
    h = (2e-9, 3e-9, 2.5e-9)
    rng = np.random.default_rng(11)
    m = rng.normal(size=(n[2], n[1], n[0], 3))
    per = O.Oracle(film(n, h, 3, pbc))
    opn = O.Oracle(film(n, h, 0, pbc))
    for axis in range(3):
        if not pbc[axis]:
            continue
        ax = 2 - axis
        Hp = per.demag_field(m.reshape(-1, 3)).reshape(m.shape)
        Hs = per.demag_field(np.roll(m, 3, axis=ax).reshape(-1, 3)).reshape(m.shape)
        assert np.abs(Hs - np.roll(Hp, 3, axis=ax)).max() < 1e-12 * MS
        # open boundaries are not shift covariant
        Ho = opn.demag_field(m.reshape(-1, 3)).reshape(m.shape)
        Hos = opn.demag_field(np.roll(m, 3, axis=ax).reshape(-1, 3)).reshape(m.shape)
        assert np.abs(Hos - np.roll(Ho, 3, axis=ax)).max() > 1e-3 * MS


def test_fft_equals_direct_periodic():
    n = (8, 6, 2)
    o = O.Oracle(film(n, (2e-9, 2e-9, 3e-9), 2, (1, 1, 0)))
    m = np.random.default_rng(5).normal(size=(n[0] * n[1] * n[2], 3))
    a = o.demag_field(m, "direct")
    b = o.demag_field(m, "fft")
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_half_period_parity_and_period():
    o = O.Oracle(film((8, 6, 1), (2e-9, 2e-9, 2e-9), 2))
    k = o.kernel(4, 1, 0)
    ref = abs(o.kernel(3, 1, 0)[3])
    # odd in x at the half period: the two minimal images cancel (to rounding)
    assert abs(k[3]) < 1e-11 * ref and abs(k[4]) < 1e-11 * ref
    assert abs(k[0]) > 0 and abs(k[2]) > 0
    k2 = o.kernel(1, 3, 0)
    assert abs(k2[3]) < 1e-11 * abs(o.kernel(1, 2, 0)[3])     # odd in y at y's half period
    for X, Y in [(3, 1), (5, 2), (4, 3), (0, 0)]:
        a = o.kernel(X, Y, 0)
        assert np.array_equal(a, o.kernel(X - 8, Y, 0))
        assert np.array_equal(a, o.kernel(X, Y + 6, 0))
    # without periodic axes the images option changes nothing; along an open
    # axis the offset is taken as it is (images only along the periodic x)
    h = (2e-9, 2e-9, 2e-9)
    q = O.Oracle(film((8, 6, 1), h, 2, (0, 0, 0)))
    assert np.array_equal(q.kernel(0, 5, 0), O.tensor(h, (0.0, 5 * h[1], 0.0)))
    p = O.Oracle(film((8, 6, 1), h, 2, (1, 0, 0)))
    want = sum(O.tensor(h, (8 * j * h[0], 5 * h[1], 0.0)) for j in range(-2, 3))
    assert np.allclose(p.kernel(0, 5, 0), want, rtol=1e-14, atol=0)


def test_uniform_film_limit():
    h = (2e-9, 2e-9, 2e-9)
    n = (16, 16, 1)
    dz, dx = [], []
    for P in (4, 8, 16):
        o = O.Oracle(film(n, h, P))
        m = np.zeros((n[0] * n[1], 3))
        m[:, 2] = 1.0
        dz.append(1.0 + o.demag_field(m, "fft")[:, 2].mean() / MS)
        m[:, 2] = 0.0
        m[:, 0] = 1.0
        dx.append(-o.demag_field(m, "fft")[:, 0].mean() / MS)
    dz, dx = np.array(dz), np.array(dx)
    assert np.all(dz > 0) and np.all(np.diff(dz) < 0) and dz[-1] < 0.01
    assert np.all(dx > 0) and np.all(np.diff(dx) < 0) and dx[-1] < 0.01
    # the finite-plate correction falls like the inverse plate width
    w = 2.0 * np.array([4, 8, 16]) + 1.0
    assert np.ptp(dz * w) < 0.15 * (dz * w).mean()
