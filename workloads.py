"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds problem statements (mesh, cell size, material, temperature,
field) and seeded random states only.  It contains none of the method's
arithmetic: no thermodynamic tables, energies, tensors or moves.  Both the CUDA
path (through ``paper_2106_05593_gb300``) and the FP64 oracle (``oracle``) read
the same dicts.

Workloads (the paper's geometries stand in as synthetic meshes, since the
paper's data are not public):
  permalloy32   32x32x1 periodic film of 5 nm cubes, no demag (Sec. II test)
  film256       256x256x1 film of 4 nm cubes with demag, field along x
                (hysteresis stand-in, Sec. III)
  chiral512     16 chains of 512x512x1 cells of 2x2x1 nm, DMI + perpendicular
                anisotropy + demag, T = 50 + 40 c K (Sec. IV)
  granular      32 uneven chains, Voronoi grains with lognormal Ms0, Ku, Tc,
                easy axes within 10 deg of z, Gaussian hotspot (Sec. III, IV)
  energy3d      256x256x4 cells of 4 nm for the differentiable energy
  probe8192     8192x8192x1 permalloy film without demag (sweep roofline probe)
"""
from __future__ import annotations

import math

import numpy as np

MUB = 9.2740100783e-24


def _base(mesh, h, **kw):
    spec = {
        "mesh": tuple(int(v) for v in mesh),
        "pbc": (False, False, False),
        "h": tuple(float(v) for v in h),
        "Ms0": 8.6e5, "A0": 1.3e-11, "D0": 0.0, "K1": 0.0, "K2": 0.0,
        "eA": (0.0, 0.0, 1.0), "Tc": 870.0, "T": 300.0, "mu": MUB,
        "B": (0.0, 0.0, 0.0), "sigma_cap": 0.03, "demag": False,
        "grain": None, "grain_exch_scale": 1.0, "aniso": "uniaxial",
    }
    spec.update(kw)
    return spec


def permalloy32(n=32):
    """Sec. II verification geometry: periodic in-plane, exchange + Zeeman only."""
    return _base((n, n, 1), (5e-9, 5e-9, 5e-9), pbc=(True, True, False),
                 B=(0.010, 0.0, 0.0))


def film256(n=256, B_mT=100.0):
    """Thin film with demag on the zero-padded grid (Sec. III)."""
    return _base((n, n, 1), (4e-9, 4e-9, 4e-9), demag=True, B=(B_mT * 1e-3, 0.0, 0.0))


def hysteresis_fields(npts=41, Bmax_mT=100.0):
    """+Bmax -> -Bmax along x in npts steps (T)."""
    return [(float(b) * 1e-3, 0.0, 0.0) for b in np.linspace(Bmax_mT, -Bmax_mT, npts)]


def chiral(n=512, T=300.0):
    """Chiral film (Sec. IV): DMI, perpendicular anisotropy, demag."""
    return _base((n, n, 1), (2e-9, 2e-9, 1e-9), Ms0=6e5, A0=1e-11, D0=1.5e-3,
                 K1=8e5, eA=(0.0, 0.0, 1.0), Tc=600.0, T=T, demag=True)


def chiral_periodic(n=512, T=300.0, images=10):
    """Chiral film (Sec. IV) periodic in the plane for exchange, DMI and the
    demag convolution (images periodic images on each side)."""
    return chiral(n, T) | {"pbc": (True, True, False), "demag_images": int(images)}


def chiral512_batch(nchains=16, n=512):
    """Temperature scan T = 50 + 40 c K, c = 0..15 (crosses Tc = 600 K)."""
    return [chiral(n, 50.0 + 40.0 * c) for c in range(nchains)]


def energy3d(n=256, nz=4):
    return _base((n, n, nz), (4e-9, 4e-9, 4e-9), Ms0=6e5, A0=1e-11, D0=1.5e-3,
                 K1=8e5, eA=(0.0, 0.0, 1.0), Tc=600.0, T=300.0, demag=True)


def probe(n=8192):
    """Sweep roofline probe: permalloy film, open edges, no demag."""
    return _base((n, n, 1), (5e-9, 5e-9, 5e-9), B=(0.010, 0.0, 0.0))


def granular_chain(n, seed, h=5e-9, grain_spacing=8e-9, Ms0=1e6, Ku=3e5, Tc=700.0,
                   sigma_ln=0.1, cap_deg=10.0, T0=300.0, Tpeak=800.0, fwhm=50e-9,
                   demag=True):
    """One granular chain: Voronoi grains (nearest of Poisson seeds at density
    1/spacing^2), per-grain lognormal Ms0, Ku, Tc (median = stated value),
    easy axis uniform on the cap of cap_deg about z, Gaussian hotspot T."""
    rng = np.random.default_rng(1000 + seed)
    L = n * h
    nseeds = max(1, rng.poisson((L / grain_spacing) ** 2))
    sx = rng.uniform(0, L, nseeds)
    sy = rng.uniform(0, L, nseeds)
    xc = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, xc, indexing="xy")          # X varies along i (fast)
    # nearest seed of every cell centre (exact nearest neighbour by k-d tree)
    from scipy.spatial import cKDTree
    _, arg = cKDTree(np.stack([sx, sy], axis=1)).query(np.stack([X.reshape(-1), Y.reshape(-1)], axis=1))
    grain = arg.astype(np.int32).reshape(n, n)
    g_Ms = Ms0 * np.exp(sigma_ln * rng.standard_normal(nseeds))
    g_Ku = Ku * np.exp(sigma_ln * rng.standard_normal(nseeds))
    g_Tc = Tc * np.exp(sigma_ln * rng.standard_normal(nseeds))
    cosmax = math.cos(math.radians(cap_deg))
    cz = 1.0 - rng.uniform(0, 1, nseeds) * (1.0 - cosmax)
    ph = rng.uniform(0, 2 * math.pi, nseeds)
    sz = np.sqrt(np.maximum(0.0, 1 - cz * cz))
    g_e = np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)
    gflat = grain.reshape(-1)
    r2 = (X - L / 2) ** 2 + (Y - L / 2) ** 2
    Tcell = T0 + (Tpeak - T0) * np.exp(-4.0 * math.log(2.0) * r2 / fwhm ** 2)
    return _base((n, n, 1), (h, h, h), Ms0=g_Ms[gflat], K1=g_Ku[gflat], eA=g_e[gflat],
                 Tc=g_Tc[gflat], T=Tcell.reshape(-1), A0=1e-11, demag=demag,
                 grain=gflat.copy(), grain_exch_scale=0.1)


def granular_sizes(nchains=32, seed=7, lo=64, hi=1024, step=2):
    """Square mesh sides drawn uniformly from the even values lo..hi (steps of
    `step`)."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.choice(np.arange(lo, hi + 1, step), size=nchains)]


def granular_batch(nchains=32, seed=7, sizes=None):
    sizes = sizes or granular_sizes(nchains, seed)
    return [granular_chain(n, c) for c, n in enumerate(sizes)]


# --------------------------------------------------------------------------- #
# seeded states


def random_state(ncell, seed, len_lo=0.8, len_hi=1.0, scale=1.0):
    """Random directions, lengths uniform in [len_lo, len_hi] * scale; float32
    values (exactly representable for both sides), shape (ncell, 4), w = 0."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((ncell, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    L = rng.uniform(len_lo, len_hi, ncell) * scale
    out = np.zeros((ncell, 4), dtype=np.float32)
    out[:, :3] = (v * L[:, None]).astype(np.float32)
    return out


def smooth_state(mesh, seed, length=0.9, tilt=0.4):
    """A slowly varying texture plus small noise (interacting-equilibrium-like)."""
    nx, ny, nz = mesh
    rng = np.random.default_rng(seed)
    k = np.indices((nz, ny, nx)).astype(np.float64)
    th = tilt * np.sin(2 * np.pi * k[2] / max(nx, 2)) * np.cos(2 * np.pi * k[1] / max(ny, 2))
    ph = 2 * np.pi * k[2] / max(nx, 2) + 0.3 * k[0]
    v = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), np.sin(th)], axis=-1).reshape(-1, 3)
    v += 0.05 * rng.standard_normal(v.shape)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    out = np.zeros((v.shape[0], 4), dtype=np.float32)
    out[:, :3] = (length * v).astype(np.float32)
    return out


def uniform_state(ncell, direction=(1.0, 0.0, 0.0), length=1.0):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    out = np.zeros((ncell, 4), dtype=np.float32)
    out[:, :3] = (length * d).astype(np.float32)
    return out
