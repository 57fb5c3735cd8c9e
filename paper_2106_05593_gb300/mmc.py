"""Python binding of the MMC library: the C-ABI calls with numpy / torch buffers.

Every step of the method runs in the library's CUDA kernels; this module only
marshals arguments (problem dicts -> C structs, arrays -> pointers).

A problem ("chain") is a dict with the keys
  mesh (nx, ny, nz), pbc (3 bools), h (3 cell sizes, m), Ms0, A0, D0, K1, K2,
  eA (3), Tc, T, mu, B (3, tesla), grain (per-cell ints or None),
  grain_exch_scale, aniso ('uniaxial' | 'cubic'), demag_images (periodic images
  per side of the demag convolution along the pbc axes; 0, the default, keeps it
  open);
Ms0, K1, eA, Tc and T may be per-cell arrays (natural order i + nx (j + ny k)).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import ChainDesc, Material, Mesh, Obs, Options, check, load

MUB = 9.2740100783e-24


def default_options(**kw) -> Options:
    """mmc_options with the library's defaults, overridden by keyword (field names
    of mmc_options in include/mmc.h, e.g. demag=1, demag_images via the problem)."""
    o = Options()
    check(load().mmc_default_options(C.byref(o)), "mmc_default_options")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def checked_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return bool(load().mmc_checked_build())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def thermo(T, Tc, V, Ms0, mu=MUB, sigma_cap=0.03):
    """The library's thermodynamic tables on the host, no GPU (Sec. II): dict of
    arrays m_e (Eq. 9), chi (Eq. 8), sigma (Eq. 13) and the Eq. 7 coefficients
    c2, c4 (F = c2 m^2 + c4 m^4 + const, J) at the temperatures T."""
    t = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    n = t.size
    out = {k: np.zeros(n) for k in ("me", "chi", "sigma", "c2", "c4")}
    check(load().mmc_thermo(_dptr(t), n, float(Tc), float(mu), float(V), float(Ms0), float(sigma_cap),
                            *[_dptr(out[k]) for k in ("me", "chi", "sigma", "c2", "c4")]), "mmc_thermo")
    return out


def demag_kernel(h, n, periodic=(0, 0, 0), images=0, offsets=None):
    """The library's demag kernel (Sec. III, Eq. 14) on the host, no GPU: an array
    (oz, oy, ox, 6) of xx yy zz xy xz yz at cell offsets 0 <= x < ox, ...
    (offsets = (ox, oy, oz), default n), periodic along the flagged axes with
    `images` images per side."""
    ox, oy, oz = n if offsets is None else offsets
    out = np.zeros(6 * ox * oy * oz)
    nn = (C.c_int * 3)(*[int(v) for v in n])
    pp = (C.c_int * 3)(*[int(bool(v)) for v in periodic])
    hh = np.ascontiguousarray(h, dtype=np.float64)
    check(load().mmc_demag_kernel(_dptr(hh), nn, pp, int(images), int(ox), int(oy), int(oz), _dptr(out)),
          "mmc_demag_kernel")
    return out.reshape(oz, oy, ox, 6)


def _percell(v, n, width=1):
    a = np.asarray(v, dtype=np.float64)
    if a.size == width:
        return None, a.reshape(width)
    return np.ascontiguousarray(a.reshape(n * width)), None


class MMC:
    """A batch of MMC chains on one GPU (a plain run is a batch of one)."""

    def __init__(self, chains, options: Options | None = None, stream=None, **opt):
        L = load()
        if isinstance(chains, dict):
            chains = [chains]
        self.specs = list(chains)
        self.nchains = len(chains)
        if options is None:
            options = default_options(**opt)
        self.options = options
        keep = []
        descs = (ChainDesc * self.nchains)()
        for k, sp in enumerate(self.specs):
            d = descs[k]
            nx, ny, nz = sp["mesh"]
            n = nx * ny * nz
            d.mesh = Mesh(nx, ny, nz, (C.c_int * 3)(*[int(bool(p)) for p in sp.get("pbc", (0, 0, 0))]),
                          int(sp.get("demag_images", 0)))
            d.cellsize = (C.c_double * 3)(*sp["h"])
            mat = Material()
            cell, val = _percell(sp["Ms0"], n)
            mat.Ms0 = float(val[0]) if val is not None else float(cell.mean())
            if cell is not None:
                keep.append(cell); mat.Ms0_cell = _dptr(cell)
            mat.A0 = float(sp.get("A0", 0.0))
            mat.D0 = float(sp.get("D0", 0.0))
            cell, val = _percell(sp.get("K1", 0.0), n)
            mat.K1 = float(val[0]) if val is not None else float(cell.mean())
            if cell is not None:
                keep.append(cell); mat.K1_cell = _dptr(cell)
            mat.K2 = float(sp.get("K2", 0.0))
            cell, val = _percell(sp.get("eA", (0.0, 0.0, 1.0)), n, 3)
            mat.e_A = (C.c_double * 3)(*(val if val is not None else (0.0, 0.0, 1.0)))
            if cell is not None:
                keep.append(cell); mat.e_A_cell = _dptr(cell)
            cell, val = _percell(sp["Tc"], n)
            mat.Tc = float(val[0]) if val is not None else float(cell.mean())
            if cell is not None:
                keep.append(cell); mat.Tc_cell = _dptr(cell)
            mat.mu_atom = float(sp.get("mu", MUB))
            mat.aniso_cubic = 1 if sp.get("aniso", "uniaxial") == "cubic" else 0
            if sp.get("grain") is not None:
                g = np.ascontiguousarray(sp["grain"], dtype=np.int32).reshape(n)
                keep.append(g)
                mat.grain = g.ctypes.data_as(C.POINTER(C.c_int))
                mat.grain_exch_scale = float(sp.get("grain_exch_scale", 1.0))
            d.material = mat
            cell, val = _percell(sp["T"], n)
            d.T = float(val[0]) if val is not None else float(cell.max())
            if cell is not None:
                keep.append(cell); d.T_cell = _dptr(cell)
            d.B = (C.c_double * 3)(*sp.get("B", (0.0, 0.0, 0.0)))
        self._ctx = C.c_void_p()
        st = None
        if stream is not None:
            st = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        check(L.mmc_create(descs, self.nchains, C.byref(options), st, C.byref(self._ctx)), "mmc_create")
        self.ncell = [int(L.mmc_ncell(self._ctx, k)) for k in range(self.nchains)]

    def close(self):
        """Release the context's device memory (mmc_destroy); idempotent."""
        if getattr(self, "_ctx", None):
            load().mmc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ state
    def set_field(self, B, chain=-1):
        """Applied field B = mu0 H (tesla, 3 components) of one chain (chain < 0: all)."""
        b = np.asarray(B, dtype=np.float64).reshape(3)
        check(load().mmc_set_field(self._ctx, int(chain), _dptr(b)), "mmc_set_field")

    def set_temperature(self, T, chain=-1, T_cell=None):
        """Temperature of one chain (chain < 0: all), kelvin; T_cell: optional
        per-cell temperatures (natural order) of one chain with per-cell tables."""
        tc = None
        if T_cell is not None:
            tc = np.ascontiguousarray(T_cell, dtype=np.float64).reshape(-1)
            assert tc.size == self.ncell[chain]
        check(load().mmc_set_temperature(self._ctx, int(chain), float(T), _dptr(tc) if tc is not None else None),
              "mmc_set_temperature")

    def set_m(self, m, chain=0):
        """m: numpy float32 (ncell, 4) on the host, or a CUDA torch tensor."""
        if hasattr(m, "is_cuda") and m.is_cuda:
            assert m.dtype.is_floating_point and m.numel() == 4 * self.ncell[chain] and m.is_contiguous()
            check(load().mmc_set_m(self._ctx, int(chain), C.c_void_p(m.data_ptr()), 1), "mmc_set_m")
            return
        a = np.ascontiguousarray(m, dtype=np.float32).reshape(-1, 4)
        assert a.shape[0] == self.ncell[chain]
        check(load().mmc_set_m(self._ctx, int(chain), a.ctypes.data_as(C.c_void_p), 0), "mmc_set_m")

    def get_m(self, chain=0, out=None):
        """m of one chain as float32 (ncell, 4) in natural order (w: grain id); into
        `out` when given (a host array or a CUDA torch tensor)."""
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            check(load().mmc_get_m(self._ctx, int(chain), C.c_void_p(out.data_ptr()), 1), "mmc_get_m")
            return out
        a = np.empty((self.ncell[chain], 4), dtype=np.float32) if out is None else out
        check(load().mmc_get_m(self._ctx, int(chain), a.ctypes.data_as(C.c_void_p), 0), "mmc_get_m")
        return a

    def set_m_all(self, m):
        """Every chain at once: m holds chain 0's cells in natural order, then chain
        1's, ... (total cells x 4 float32), on the host or as a CUDA torch tensor."""
        tot = int(sum(self.ncell))
        if hasattr(m, "is_cuda") and m.is_cuda:
            assert m.dtype.is_floating_point and m.numel() == 4 * tot and m.is_contiguous()
            check(load().mmc_set_m_all(self._ctx, C.c_void_p(m.data_ptr()), 1), "mmc_set_m_all")
            return
        a = np.ascontiguousarray(m, dtype=np.float32).reshape(-1, 4)
        assert a.shape[0] == tot
        check(load().mmc_set_m_all(self._ctx, a.ctypes.data_as(C.c_void_p), 0), "mmc_set_m_all")

    def get_m_all(self, out=None):
        """Every chain's m, concatenated in chain order (total cells x 4 float32)."""
        tot = int(sum(self.ncell))
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            check(load().mmc_get_m_all(self._ctx, C.c_void_p(out.data_ptr()), 1), "mmc_get_m_all")
            return out
        a = np.empty((tot, 4), dtype=np.float32) if out is None else out
        check(load().mmc_get_m_all(self._ctx, a.ctypes.data_as(C.c_void_p), 0), "mmc_get_m_all")
        return a

    def init_random(self, seed, length=0.0):
        """Random directions for every chain (Philox counter (cell, 0, chain, 1));
        |m| = length, or m_e (the Eq. 7 rms length where m_e = 0) when length <= 0."""
        check(load().mmc_init_random(self._ctx, int(seed), float(length)), "mmc_init_random")

    # ------------------------------------------------------------------ MC
    def sweep(self, n, seed):
        """n MMC iterations of every chain (Sec. II): demag update, red pass, black
        pass (per the options), cone adaptation every 100 iterations."""
        check(load().mmc_sweep(self._ctx, int(n), int(seed)), "mmc_sweep")

    def sweep_serial(self, n, seed):
        """n iterations of the serial exact-demag form (App. B): cells in index
        order, demag field updated after every accepted move."""
        check(load().mmc_sweep_serial(self._ctx, int(n), int(seed)), "mmc_sweep_serial")

    def minimize(self, chain=0, maxit=20000, tol=1e-5):
        """Zero-temperature steepest descent of one chain (the paper's SDesc,
        Sec. III); the chain's state becomes the result.  Returns a dict with
        the steps taken, the final largest normalized torque and the energy
        terms of the result."""
        it = C.c_int64(0)
        tq = np.zeros(1)
        E = np.zeros(7)
        check(load().mmc_minimize(self._ctx, int(chain), int(maxit), float(tol), C.byref(it), _dptr(tq), _dptr(E)),
              "mmc_minimize")
        return {"iters": int(it.value), "torque": float(tq[0]), "converged": bool(tq[0] < tol),
                "energy": E.copy()}

    def sweep_sampled(self, n, seed, every):
        """Like sweep, accumulating an observables snapshot every `every` iterations."""
        check(load().mmc_sweep_sampled(self._ctx, int(n), int(seed), int(every)), "mmc_sweep_sampled")

    def demag_update(self):
        """Recompute the demag field (Eq. 14) of every chain from the current state."""
        check(load().mmc_demag_update(self._ctx), "mmc_demag_update")

    def pass_debug(self, chain, color, sweep, seed, theta_deg):
        """One sublattice pass of one chain with explicit iteration index and cone
        angle; returns the FP32 decision values and accept flags per cell (natural
        order; -1 for cells of the other colour).  The state is updated."""
        n = self.ncell[chain]
        dec = np.zeros(n, dtype=np.float32)
        acc = np.zeros(n, dtype=np.int8)
        check(load().mmc_pass_debug(self._ctx, int(chain), int(color), int(sweep), int(seed),
                                    float(theta_deg), dec.ctypes.data_as(C.c_void_p),
                                    acc.ctypes.data_as(C.c_void_p)), "mmc_pass_debug")
        return dec, acc

    # ------------------------------------------------------------------ measurements
    def observables(self, chain=0, reset=False):
        """Averages over the accumulated snapshots, or over the current state when
        there are none: <m>, <|m|>, <|m|^2>, |m| histogram, acceptance rate of the
        last window, cone angle, iteration count, non-finite count."""
        bins = self.options.hist_bins
        hist = np.zeros(bins + 1, dtype=np.int64)
        o = Obs()
        o.hist = hist.ctypes.data_as(C.POINTER(C.c_int64))
        check(load().mmc_observables(self._ctx, int(chain), C.byref(o), int(bool(reset))), "mmc_observables")
        return {"mean_m": np.array(o.mean_m[:]), "mean_len": o.mean_len, "mean_len2": o.mean_len2,
                "nsnap": o.nsnap, "nonfinite": o.nonfinite, "acc_rate": o.acc_rate,
                "theta_deg": o.theta_deg, "sweeps": o.sweeps, "hist": hist}

    def observables_all(self, reset=False):
        """observables() of every chain, read in one device round trip."""
        bins = self.options.hist_bins
        n = self.nchains
        hist = np.zeros((n, bins + 1), dtype=np.int64)
        obs = (Obs * n)()
        for k in range(n):
            obs[k].hist = hist[k].ctypes.data_as(C.POINTER(C.c_int64))
        check(load().mmc_observables_all(self._ctx, obs, int(bool(reset))), "mmc_observables_all")
        return [{"mean_m": np.array(o.mean_m[:]), "mean_len": o.mean_len, "mean_len2": o.mean_len2,
                 "nsnap": o.nsnap, "nonfinite": o.nonfinite, "acc_rate": o.acc_rate,
                 "theta_deg": o.theta_deg, "sweeps": o.sweeps, "hist": hist[k]} for k, o in enumerate(obs)]

    def check_report(self, clear=False):
        """Bounds-checked builds: out-of-range indices met so far, and the first
        (site name, index, [lo, hi)); always zero in normal builds."""
        n = C.c_int64(0)
        site = C.c_int(0)
        rng = (C.c_int64 * 3)()
        check(load().mmc_check_report(self._ctx, C.byref(n), C.byref(site), rng, int(bool(clear))),
              "mmc_check_report")
        return {"count": int(n.value), "site": load().mmc_check_site_name(site.value).decode(),
                "index": int(rng[0]), "lo": int(rng[1]), "hi": int(rng[2])}

    def energy(self, chain=0):
        """Energy terms of the current state (J): total, exchange, DMI, anisotropy,
        Zeeman, longitudinal, demag (FP64 convolution)."""
        out = np.zeros(7)
        check(load().mmc_energy(self._ctx, int(chain), _dptr(out)), "mmc_energy")
        return out

    def demag_field(self, chain=0):
        """Demag field H_d (A/m) of the current state, FP64 convolution, (ncell, 3)."""
        H = np.zeros(3 * self.ncell[chain])
        check(load().mmc_demag_field(self._ctx, int(chain), _dptr(H)), "mmc_demag_field")
        return H.reshape(-1, 3)

    def sweep_field(self, chain=0):
        """Demag field H_d (A/m) the sweep uses (the context's own convolution:
        FP32 unless demag_fp64, the picked FFT variant), (ncell, 3)."""
        H = np.zeros(3 * self.ncell[chain])
        check(load().mmc_sweep_field(self._ctx, int(chain), _dptr(H)), "mmc_sweep_field")
        return H.reshape(-1, 3)

    def angle_hist(self, chain=0, bins=100, lo=0.0, hi=np.pi):
        """Angular-deviation histogram of the current state (Sec. II, Fig. 1d-f):
        (counts, bins + 1 entries with the out-of-range angles last; mean direction)."""
        h = np.zeros(bins + 1, dtype=np.int64)
        d = np.zeros(3)
        check(load().mmc_angle_hist(self._ctx, int(chain), int(bins), float(lo), float(hi),
                                    h.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(d)), "mmc_angle_hist")
        return h, d

    def trial_terms(self, chain=0, sweep=0, seed=1, theta_deg=-1.0):
        """App. B (Fig. 11): mean |dF| / kT per term of the trial moves of every cell
        at the current state -- [exchange, DMI, anisotropy, Zeeman, longitudinal,
        demag] -- for the moves of iteration `sweep` with `seed` (theta_deg < 0:
        the chain's current cone angle)."""
        out = np.zeros(6)
        check(load().mmc_trial_terms(self._ctx, int(chain), int(sweep), int(seed), float(theta_deg), _dptr(out)),
              "mmc_trial_terms")
        return out

    def tables(self, chain=0):
        """Per-cell m_e(T), chi(T) (Eqs. 8-9) and the length-move width sigma (Eq. 13)."""
        n = self.ncell[chain]
        me, chi, sg = np.zeros(n), np.zeros(n), np.zeros(n)
        check(load().mmc_tables(self._ctx, int(chain), _dptr(me), _dptr(chi), _dptr(sg)), "mmc_tables")
        return {"me": me, "chi": chi, "sigma": sg}

    def energy_grad(self, m, params=None, chain=0, grad=True):
        """Differentiable form: m is a CUDA torch tensor (ncell, 3), float32 or
        float64; params = (Ms0, A0, D0, Ku, chi) or None.  Returns (E[7],
        dE/dm tensor or None, dE/dparams[5])."""
        import torch
        assert m.is_cuda and m.is_contiguous() and m.shape == (self.ncell[chain], 3)
        fp64 = m.dtype == torch.float64
        assert fp64 or m.dtype == torch.float32
        E = np.zeros(7)
        dp = np.zeros(5)
        pp = None
        if params is not None:
            pa = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(5))
            pp = _dptr(pa)
        g = torch.empty_like(m) if grad else None
        torch.cuda.current_stream(m.device).synchronize()
        check(load().mmc_energy_grad(self._ctx, int(chain), C.c_void_p(m.data_ptr()), int(fp64), pp,
                                     _dptr(E), C.c_void_p(g.data_ptr()) if grad else None, _dptr(dp)),
              "mmc_energy_grad")
        return E, g, dp

    def phase_times(self, n, seed):
        """n iterations eagerly with CUDA events around every kernel: returns
        {kind: (total ms, launches)} for the eight kernel kinds."""
        ms = np.zeros(8)
        cnt = np.zeros(8, dtype=np.int64)
        check(load().mmc_phase_times(self._ctx, int(n), int(seed), _dptr(ms),
                                     cnt.ctypes.data_as(C.POINTER(C.c_int64))), "mmc_phase_times")
        kinds = ("demag_rows_fwd", "demag_cols", "demag_rows_inv", "sweep_pass", "observables", "advance",
                 "black_pass_rows_fwd", "rows_inv_red_pass")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(kinds)}

    def fft_tuning(self):
        """(variant, create-time ms of variants 1, 2, 3, 4) of the FP32 2D demag kernels."""
        v = C.c_int(0)
        ms = np.zeros(4)
        check(load().mmc_fft_tuning(self._ctx, C.byref(v), _dptr(ms)), "mmc_fft_tuning")
        return int(v.value), tuple(float(x) for x in ms)

    def tuning(self):
        """The create-time autotuner's picks: dict with fft_variant, stream_groups,
        from_cache and the timed ms per update (FFT variants 1..4) and per
        iteration (1, 2, 3 groups)."""
        v, gr, fc = C.c_int(0), C.c_int(0), C.c_int(0)
        ms = np.zeros(7)
        check(load().mmc_tuning(self._ctx, C.byref(v), C.byref(gr), C.byref(fc), _dptr(ms)), "mmc_tuning")
        return {"fft_variant": int(v.value), "stream_groups": int(gr.value), "from_cache": bool(fc.value),
                "fft_ms": tuple(float(x) for x in ms[:4]), "groups_ms": tuple(float(x) for x in ms[4:])}

    @property
    def launches(self) -> int:
        """Kernels the context has launched (graph replays counted per kernel)."""
        return int(load().mmc_kernel_launches(self._ctx))

    def checkpoint(self) -> bytes:
        """The whole mutable state (moments, per-chain counters, cone angles, sweep
        counter) as bytes; restore() on a context of the same problem resumes it
        bit for bit."""
        L = load()
        n = C.c_size_t(0)
        check(L.mmc_checkpoint(self._ctx, None, C.byref(n)), "mmc_checkpoint")
        buf = (C.c_char * n.value)()
        check(L.mmc_checkpoint(self._ctx, buf, C.byref(n)), "mmc_checkpoint")
        return bytes(buf)

    def restore(self, data: bytes):
        """Resume a checkpoint taken on a context of the same problem."""
        buf = C.create_string_buffer(data, len(data))
        check(load().mmc_restore(self._ctx, buf, len(data)), "mmc_restore")
