"""FP64 serial CPU oracle of the micromagnetic Monte Carlo method (arXiv:2106.05593).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are its only users; the product package never
imports it.  The arithmetic lives in ``mmc_oracle.c`` (plain C, FP64, one thread);
this module is argument marshalling around it (ctypes + numpy).

Each wrapped function names the paper passage it follows (Sec. II Eqs. 1-13,
Sec. III Eq. 14, Sec. IV Eq. 15, App. B).  What pins each function is listed in
the header of ``mmc_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "mmc_oracle.c")
_lock = threading.Lock()

KB = 1.380649e-23
MUB = 9.2740100783e-24
MU0 = 1.25663706212e-6


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, no fast-math, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)
                and os.path.getmtime(_SO) >= os.path.getmtime(os.path.join(_HERE, "mmc_oracle.h"))):
            return _SO
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("pbc", C.c_int * 3),
        ("h", C.c_double * 3),
        ("A0", C.c_double), ("D0", C.c_double), ("mu", C.c_double),
        ("sigma_cap", C.c_double), ("grain_exch_scale", C.c_double),
        ("B", C.c_double * 3),
        ("demag", C.c_int), ("demag_self", C.c_int), ("len_power", C.c_int),
        ("aniso_cubic", C.c_int),
        ("Ms0", C.POINTER(C.c_double)), ("K1", C.POINTER(C.c_double)),
        ("K2", C.POINTER(C.c_double)), ("eA", C.POINTER(C.c_double)),
        ("Tc", C.POINTER(C.c_double)), ("T", C.POINTER(C.c_double)),
        ("grain", C.POINTER(C.c_int)), ("cell_base", C.c_uint32),
        ("demag_images", C.c_int),
    ]


class _Obs(C.Structure):
    _fields_ = [
        ("sum_m", C.c_double * 3), ("sum_len", C.c_double), ("sum_len2", C.c_double),
        ("nsamples", C.c_int64), ("nsnap", C.c_int64),
        ("hist", C.POINTER(C.c_int64)), ("hist_bins", C.c_int), ("hist_max", C.c_double),
    ]


class RunState(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("chain", C.c_uint32), ("sweep", C.c_uint32),
        ("theta_deg", C.c_double), ("win_acc", C.c_int64), ("win_att", C.c_int64),
        ("adapt", C.c_int), ("demag_mode", C.c_int), ("stripes", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        dp = C.POINTER(C.c_double)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_u01.restype = C.c_double
        L.orc_u01.argtypes = [C.c_uint32]
        for name in ("orc_langevin", "orc_langevin_d"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double]
        L.orc_me.restype = C.c_double
        L.orc_me.argtypes = [C.c_double, C.c_double]
        L.orc_chi.restype = C.c_double
        L.orc_chi.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_sigma.restype = C.c_double
        L.orc_sigma.argtypes = [C.c_double] * 6
        L.orc_long_energy.restype = C.c_double
        L.orc_long_energy.argtypes = [C.c_double] * 6
        L.orc_newell.argtypes = [C.c_double] * 6 + [dp]
        L.orc_tensor_quad.argtypes = [C.c_double] * 6 + [C.c_int, dp]
        L.orc_tensor.argtypes = [C.c_double] * 6 + [dp]
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Problem)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_ncell.restype = C.c_int
        L.orc_ncell.argtypes = [C.c_void_p]
        L.orc_set_field.argtypes = [C.c_void_p, dp]
        L.orc_tables.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        L.orc_demag_field.argtypes = [C.c_void_p, dp, dp, C.c_int]
        L.orc_kernel.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, dp]
        L.orc_energy.argtypes = [C.c_void_p, dp, dp]
        L.orc_pervector_sums.argtypes = [C.c_void_p, dp, dp]
        L.orc_local_dF.argtypes = [C.c_void_p, dp, dp, C.c_int, dp, dp]
        L.orc_energy_grad.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_pass.restype = C.c_int64
        L.orc_pass.argtypes = [C.c_void_p, dp, dp, C.c_int, C.c_uint32, C.c_uint32, C.c_uint64,
                               C.c_double, C.POINTER(C.c_int8), dp, dp]
        L.orc_trial_terms.argtypes = [C.c_void_p, dp, dp, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double, dp]
        L.orc_angle_hist.argtypes = [C.c_void_p, dp, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_int64), dp]
        L.orc_sdesc.restype = C.c_int
        L.orc_sdesc.argtypes = [C.c_void_p, dp, C.c_int, C.c_double, C.POINTER(C.c_int), dp]
        L.orc_serial_sweep.restype = C.c_int64
        L.orc_serial_sweep.argtypes = [C.c_void_p, dp, dp, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double]
        L.orc_run.restype = C.c_int64
        L.orc_run.argtypes = [C.c_void_p, dp, C.c_int64, C.POINTER(RunState), C.POINTER(_Obs), C.c_int]
        L.orc_obs_accumulate.argtypes = [C.c_void_p, dp, C.POINTER(_Obs)]
        L.orc_hist.argtypes = [dp, C.c_int64, C.c_int, C.c_double, C.POINTER(C.c_int64)]
        L.orc_adapt_theta.restype = C.c_double
        L.orc_adapt_theta.argtypes = [C.c_double, C.c_int64, C.c_int64]
        L.orc_init_state.argtypes = [C.c_void_p, dp, C.c_int, dp, C.c_double, C.c_uint32, C.c_uint64]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------------------- #
# free functions


def philox(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) of one 128-bit counter."""
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u01(r):
    """((r >> 9) + 1/2) * 2^-23."""
    return lib().orc_u01(int(r) & 0xFFFFFFFF)


def langevin(x):
    return lib().orc_langevin(float(x))


def langevin_d(x):
    return lib().orc_langevin_d(float(x))


def me(T, Tc):
    """Eq. 9 (zero field)."""
    return lib().orc_me(float(T), float(Tc))


def chi(T, Tc, mu=MUB):
    """Eq. 8, in 1/T."""
    return lib().orc_chi(float(T), float(Tc), float(mu))


def sigma(T, Tc, V, Ms0, mu=MUB, cap=0.03):
    """Eq. 13 with the cap."""
    return lib().orc_sigma(float(T), float(Tc), float(mu), float(V), float(Ms0), float(cap))


def long_energy(m, T, Tc, V, Ms0, mu=MUB):
    """Exponent of Eq. 7 times kT (J)."""
    return lib().orc_long_energy(float(m), float(T), float(Tc), float(mu), float(V), float(Ms0))


def newell(h, R):
    out = np.zeros(6)
    lib().orc_newell(*[float(v) for v in h], *[float(v) for v in R], _dp(out))
    return out


def tensor_quad(h, R, npts=5):
    out = np.zeros(6)
    lib().orc_tensor_quad(*[float(v) for v in h], *[float(v) for v in R], int(npts), _dp(out))
    return out


def tensor(h, R):
    out = np.zeros(6)
    lib().orc_tensor(*[float(v) for v in h], *[float(v) for v in R], _dp(out))
    return out


def adapt_theta(theta, acc, att):
    return lib().orc_adapt_theta(float(theta), int(acc), int(att))


def hist(m, bins=200, hmax=1.0):
    """|m| histogram of a state (Sec. II, Figs. 1-2), FP64: `bins` equal bins on
    [0, hmax) and the lengths at or beyond hmax in the last of bins + 1 entries."""
    mm = np.ascontiguousarray(np.asarray(m, dtype=np.float64)[..., :3]).reshape(-1)
    h = np.zeros(bins + 1, dtype=np.int64)
    lib().orc_hist(_dp(mm), mm.size // 3, int(bins), float(hmax), h.ctypes.data_as(C.POINTER(C.c_int64)))
    return h


# --------------------------------------------------------------------------- #
# problem context


def _cell_array(v, n, width=1):
    a = np.asarray(v, dtype=np.float64)
    if a.size == width:
        a = np.broadcast_to(a.reshape(1, width), (n, width))
    return np.ascontiguousarray(a.reshape(n * width) if width > 1 else a.reshape(n))


class Oracle:
    """One problem (Sec. II-IV statement): mesh, cell size, material, T, field.

    ``spec`` is a plain dict (see ``workloads.py``):
      mesh (nx, ny, nz), pbc (3 bools), h (3 floats, m), Ms0, A0, D0, K1, K2, eA,
      Tc, T (scalars or per-cell arrays), mu, B (T), sigma_cap, demag,
      grain (per-cell int or None), grain_exch_scale, aniso ('uniaxial'|'cubic'),
      demag_images (periodic demag images per side along the pbc axes; 0 open).
    """

    def __init__(self, spec, len_power=4, demag_self=False):
        L = lib()
        nx, ny, nz = spec["mesh"]
        n = nx * ny * nz
        self.n = n
        self.spec = spec
        self._keep = {
            "Ms0": _cell_array(spec["Ms0"], n),
            "K1": _cell_array(spec.get("K1", 0.0), n),
            "K2": _cell_array(spec.get("K2", 0.0), n),
            "eA": _cell_array(spec.get("eA", (0.0, 0.0, 1.0)), n, 3),
            "Tc": _cell_array(spec["Tc"], n),
            "T": _cell_array(spec["T"], n),
        }
        grain = spec.get("grain")
        self._grain = None if grain is None else np.ascontiguousarray(grain, dtype=np.int32).reshape(n)
        p = _Problem()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.pbc = (C.c_int * 3)(*[int(bool(v)) for v in spec.get("pbc", (0, 0, 0))])
        p.h = (C.c_double * 3)(*spec["h"])
        p.A0 = spec.get("A0", 0.0)
        p.D0 = spec.get("D0", 0.0)
        p.mu = spec.get("mu", MUB)
        p.sigma_cap = spec.get("sigma_cap", 0.03)
        p.grain_exch_scale = spec.get("grain_exch_scale", 1.0)
        p.B = (C.c_double * 3)(*spec.get("B", (0.0, 0.0, 0.0)))
        p.demag = int(bool(spec.get("demag", False)))
        p.demag_self = int(bool(demag_self))
        p.len_power = int(len_power)
        p.cell_base = int(spec.get("cell_base", 0))
        p.demag_images = int(spec.get("demag_images", 0))
        p.aniso_cubic = 1 if spec.get("aniso", "uniaxial") == "cubic" else 0
        for k in ("Ms0", "K1", "K2", "eA", "Tc", "T"):
            setattr(p, k, _dp(self._keep[k]))
        p.grain = self._grain.ctypes.data_as(C.POINTER(C.c_int)) if self._grain is not None else None
        self._ctx = L.orc_create(C.byref(p))
        self.V = spec["h"][0] * spec["h"][1] * spec["h"][2]

    def __del__(self):
        if getattr(self, "_ctx", None):
            lib().orc_destroy(self._ctx)
            self._ctx = None

    @staticmethod
    def _m(m):
        return np.ascontiguousarray(np.asarray(m, dtype=np.float64)[..., :3]).reshape(-1)

    def set_field(self, B):
        b = np.asarray(B, dtype=np.float64)
        lib().orc_set_field(self._ctx, _dp(b))

    def tables(self):
        n = self.n
        out = [np.zeros(n) for _ in range(5)]
        lib().orc_tables(self._ctx, *[_dp(a) for a in out])
        return dict(zip(("me", "chi", "sigma", "K1T", "K2T"), out))

    def kernel(self, X, Y, Z):
        """Demag kernel at cell offset (X, Y, Z): the Newell tensor, or along
        periodic demag axes its truncated sum over images (Sec. III films);
        [xx, yy, zz, xy, xz, yz]."""
        out = np.zeros(6)
        lib().orc_kernel(self._ctx, int(X), int(Y), int(Z), _dp(out))
        return out

    def demag_field(self, m, method="direct"):
        """Eq. 14 field (A/m), shape (n, 3)."""
        mm = self._m(m)
        H = np.zeros(3 * self.n)
        lib().orc_demag_field(self._ctx, _dp(mm), _dp(H), 0 if method == "direct" else 1)
        return H.reshape(self.n, 3)

    def energy(self, m):
        """[total, exchange, dmi, anisotropy, zeeman, longitudinal, demag] (J)."""
        mm = self._m(m)
        out = np.zeros(7)
        lib().orc_energy(self._ctx, _dp(mm), _dp(out))
        return out

    def pervector_sums(self, m):
        mm = self._m(m)
        out = np.zeros(3)
        lib().orc_pervector_sums(self._ctx, _dp(mm), _dp(out))
        return out

    def local_dF(self, m, H, i, mnew):
        mm = self._m(m)
        Hh = np.ascontiguousarray(H, dtype=np.float64).reshape(-1) if H is not None else np.zeros(3 * self.n)
        mn = np.ascontiguousarray(mnew, dtype=np.float64).reshape(3)
        out = np.zeros(7)
        lib().orc_local_dF(self._ctx, _dp(mm), _dp(Hh), int(i), _dp(mn), _dp(out))
        return out

    def energy_grad(self, m):
        mm = self._m(m)
        g = np.zeros(3 * self.n)
        dp = np.zeros(5)
        E = np.zeros(7)
        lib().orc_energy_grad(self._ctx, _dp(mm), _dp(g), _dp(dp), _dp(E))
        return g.reshape(self.n, 3), dp, E

    def sweep_pass(self, m, H, color, sweep, chain, seed, theta_deg):
        """One sublattice pass; returns (m_new (n,3), acc int8, dec, band)."""
        mm = self._m(m).copy()
        n = self.n
        Hh = (np.ascontiguousarray(H, dtype=np.float64).reshape(-1) if H is not None
              else np.zeros(3 * n))
        acc = np.zeros(n, dtype=np.int8)
        dec = np.zeros(n)
        band = np.zeros(n)
        lib().orc_pass(self._ctx, _dp(mm), _dp(Hh), int(color), int(sweep), int(chain), int(seed),
                       float(theta_deg), acc.ctypes.data_as(C.POINTER(C.c_int8)), _dp(dec), _dp(band))
        return mm.reshape(n, 3), acc, dec, band

    def serial_sweep(self, m, H, sweep, chain, seed, theta_deg):
        mm = self._m(m).copy()
        Hh = np.ascontiguousarray(H, dtype=np.float64).reshape(-1).copy()
        nacc = lib().orc_serial_sweep(self._ctx, _dp(mm), _dp(Hh), int(sweep), int(chain),
                                      int(seed), float(theta_deg))
        return mm.reshape(self.n, 3), Hh.reshape(self.n, 3), nacc

    def trial_terms(self, m, H, sweep, chain, seed, theta_deg):
        """App. B (Fig. 11): mean |dF_term| / kT over the trial moves of every cell
        at state m (frozen field H, or None for the field of m):
        [ex, dmi, an, zee, long, demag]."""
        mm = self._m(m)
        if H is None:
            H = self.demag_field(mm.reshape(-1, 3), "direct" if self.n <= 4096 else "fft")
        Hf = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(-1))
        out = np.zeros(6)
        lib().orc_trial_terms(self._ctx, _dp(mm), _dp(Hf), int(sweep), int(chain), int(seed),
                              float(theta_deg), _dp(out))
        return out

    def angle_hist(self, m, bins=100, lo=0.0, hi=np.pi):
        """Histogram of the polar angle to the mean direction (Sec. II, Fig. 1d-f):
        (counts of bins + 1 entries, the last for angles outside [lo, hi), mean direction)."""
        mm = self._m(m)
        h = np.zeros(bins + 1, dtype=np.int64)
        d = np.zeros(3)
        lib().orc_angle_hist(self._ctx, _dp(mm), int(bins), float(lo), float(hi),
                             h.ctypes.data_as(C.POINTER(C.c_int64)), _dp(d))
        return h, d

    def sdesc(self, m, maxit=20000, tol=1e-5):
        """Zero-temperature steepest descent (Sec. III SDesc) from m; returns
        (m_min (n, 3), converged, iterations, final max normalized torque)."""
        mm = self._m(m).copy()
        it = C.c_int(0)
        tq = np.zeros(1)
        rc = lib().orc_sdesc(self._ctx, _dp(mm), int(maxit), float(tol), C.byref(it), _dp(tq))
        return mm.reshape(self.n, 3), rc == 0, int(it.value), float(tq[0])

    def init_state(self, random=False, direction=(1.0, 0.0, 0.0), length=1.0, chain=0, seed=1):
        m = np.zeros(3 * self.n)
        d = np.asarray(direction, dtype=np.float64)
        lib().orc_init_state(self._ctx, _dp(m), int(bool(random)), _dp(d), float(length),
                             int(chain), int(seed))
        return m.reshape(self.n, 3)

    def run(self, m, nsweeps, state: RunState, obs_every=0, hist_bins=200, hist_max=1.0):
        """n full sweeps (Sec. II); returns (m, accepted, obs dict or None)."""
        mm = self._m(m).copy()
        obs_p = None
        hist = None
        if obs_every > 0:
            hist = np.zeros(hist_bins + 1, dtype=np.int64)
            ob = _Obs()
            ob.hist = hist.ctypes.data_as(C.POINTER(C.c_int64))
            ob.hist_bins = hist_bins
            ob.hist_max = hist_max
            obs_p = C.byref(ob)
        nacc = lib().orc_run(self._ctx, _dp(mm), int(nsweeps), C.byref(state), obs_p, int(obs_every))
        obs = None
        if obs_every > 0:
            ns = max(ob.nsamples, 1)
            obs = {"mean_m": np.array(ob.sum_m[:]) / ns, "mean_len": ob.sum_len / ns,
                   "mean_len2": ob.sum_len2 / ns, "hist": hist, "nsnap": ob.nsnap,
                   "nsamples": ob.nsamples}
        return mm.reshape(self.n, 3), nacc, obs


def new_state(seed=1, chain=0, theta_deg=30.0, adapt=True, demag_mode=1, sweep=0, stripes=1):
    st = RunState()
    st.seed = seed
    st.chain = chain
    st.sweep = sweep
    st.theta_deg = theta_deg
    st.win_acc = 0
    st.win_att = 0
    st.adapt = int(bool(adapt))
    st.demag_mode = demag_mode
    st.stripes = int(stripes)
    return st
