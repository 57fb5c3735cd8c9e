"""ctypes declarations of the C ABI in include/mmc.h (argument marshalling only).

The shared library is loaded from this package directory; a missing library is
an error (there is no fallback implementation).  MMC_LIB_VARIANT=checked loads
the bounds-checked build (libmmc_checked.so) instead.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmc_checked.so" if os.environ.get("MMC_LIB_VARIANT") == "checked"
                        else "libmmc.so")

MMC_OK = 0
STATUS = {0: "MMC_OK", -1: "MMC_ERR_ARG", -2: "MMC_ERR_CUDA", -3: "MMC_ERR_TIMEOUT",
          -4: "MMC_ERR_NONFINITE", -5: "MMC_ERR_UNSUPPORTED", -6: "MMC_ERR_NOMEM"}

# every function declared in include/mmc.h
EXPORTS = [
    "mmc_default_options", "mmc_create", "mmc_create_single", "mmc_destroy", "mmc_set_field",
    "mmc_set_m", "mmc_get_m", "mmc_set_m_all", "mmc_get_m_all", "mmc_observables_all", "mmc_init_random", "mmc_sweep", "mmc_sweep_sampled",
    "mmc_demag_update", "mmc_pass_debug", "mmc_observables", "mmc_energy", "mmc_demag_field",
    "mmc_tables", "mmc_energy_grad", "mmc_phase_times", "mmc_fft_tuning", "mmc_tuning", "mmc_sweep_field", "mmc_sweep_serial", "mmc_minimize", "mmc_set_temperature", "mmc_angle_hist", "mmc_trial_terms", "mmc_kernel_launches", "mmc_nchains", "mmc_ncell", "mmc_demag_kernel", "mmc_thermo",
    "mmc_checkpoint", "mmc_restore", "mmc_observables_noalloc", "mmc_checked_build", "mmc_check_report", "mmc_check_total",
    "mmc_check_site_name", "mmc_status_str", "mmc_last_error",
]


class MmcError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("periodic", C.c_int * 3),
                ("demag_images", C.c_int)]


class Material(C.Structure):
    _fields_ = [
        ("Ms0", C.c_double), ("A0", C.c_double), ("D0", C.c_double), ("K1", C.c_double),
        ("K2", C.c_double), ("e_A", C.c_double * 3), ("Tc", C.c_double), ("mu_atom", C.c_double),
        ("aniso_cubic", C.c_int),
        ("Ms0_cell", C.POINTER(C.c_double)), ("K1_cell", C.POINTER(C.c_double)),
        ("e_A_cell", C.POINTER(C.c_double)), ("Tc_cell", C.POINTER(C.c_double)),
        ("grain", C.POINTER(C.c_int)), ("grain_exch_scale", C.c_double),
    ]


class Options(C.Structure):
    _fields_ = [
        ("demag", C.c_int), ("demag_per_pass", C.c_int), ("demag_fp64", C.c_int),
        ("demag_cufft", C.c_int), ("adapt", C.c_int), ("theta0_deg", C.c_double),
        ("sigma_cap", C.c_double), ("hist_bins", C.c_int), ("hist_max", C.c_double),
        ("use_graphs", C.c_int), ("stream_groups", C.c_int), ("demag_self", C.c_int), ("fft_variant", C.c_int),
        ("demag_stripes", C.c_int), ("chain_base", C.c_int),
        ("sweep_tiles", C.c_int), ("wait_polls", C.c_int), ("wait_test", C.c_int), ("fuse_passes", C.c_int),
    ]


class ChainDesc(C.Structure):
    _fields_ = [("mesh", Mesh), ("cellsize", C.c_double * 3), ("material", Material),
                ("T", C.c_double), ("T_cell", C.POINTER(C.c_double)), ("B", C.c_double * 3)]


class Obs(C.Structure):
    _fields_ = [("mean_m", C.c_double * 3), ("mean_len", C.c_double), ("mean_len2", C.c_double),
                ("nsnap", C.c_int64), ("nonfinite", C.c_int64), ("acc_rate", C.c_double),
                ("theta_deg", C.c_double), ("sweeps", C.c_int64), ("hist", C.POINTER(C.c_int64))]


_lib = None


def load():
    """Load libmmc.so (built by paper_2106_05593_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2106_05593_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    st = C.c_int
    vp = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.mmc_default_options.restype = st
    L.mmc_default_options.argtypes = [C.POINTER(Options)]
    L.mmc_create.restype = st
    L.mmc_create.argtypes = [C.POINTER(ChainDesc), C.c_int, C.POINTER(Options), vp, C.POINTER(vp)]
    L.mmc_create_single.restype = st
    L.mmc_create_single.argtypes = [C.POINTER(Mesh), dp, C.POINTER(Material), C.c_double, dp,
                                    C.POINTER(Options), vp, C.POINTER(vp)]
    L.mmc_destroy.restype = None
    L.mmc_destroy.argtypes = [vp]
    L.mmc_set_field.restype = st
    L.mmc_set_field.argtypes = [vp, C.c_int, dp]
    L.mmc_set_m.restype = st
    L.mmc_set_m.argtypes = [vp, C.c_int, vp, C.c_int]
    L.mmc_get_m.restype = st
    L.mmc_get_m.argtypes = [vp, C.c_int, vp, C.c_int]
    L.mmc_set_m_all.restype = st
    L.mmc_set_m_all.argtypes = [vp, vp, C.c_int]
    L.mmc_get_m_all.restype = st
    L.mmc_get_m_all.argtypes = [vp, vp, C.c_int]
    L.mmc_init_random.restype = st
    L.mmc_init_random.argtypes = [vp, C.c_uint64, C.c_double]
    L.mmc_sweep.restype = st
    L.mmc_sweep.argtypes = [vp, C.c_int64, C.c_uint64]
    L.mmc_sweep_sampled.restype = st
    L.mmc_sweep_sampled.argtypes = [vp, C.c_int64, C.c_uint64, C.c_int]
    L.mmc_demag_update.restype = st
    L.mmc_demag_update.argtypes = [vp]
    L.mmc_pass_debug.restype = st
    L.mmc_pass_debug.argtypes = [vp, C.c_int, C.c_int, C.c_uint32, C.c_uint64, C.c_double, vp, vp]
    L.mmc_observables.restype = st
    L.mmc_observables.argtypes = [vp, C.c_int, C.POINTER(Obs), C.c_int]
    L.mmc_observables_all.restype = st
    L.mmc_observables_all.argtypes = [vp, C.POINTER(Obs), C.c_int]
    L.mmc_energy.restype = st
    L.mmc_energy.argtypes = [vp, C.c_int, dp]
    L.mmc_demag_field.restype = st
    L.mmc_demag_field.argtypes = [vp, C.c_int, dp]
    L.mmc_sweep_field.restype = st
    L.mmc_sweep_field.argtypes = [vp, C.c_int, dp]
    L.mmc_tables.restype = st
    L.mmc_tables.argtypes = [vp, C.c_int, dp, dp, dp]
    L.mmc_energy_grad.restype = st
    L.mmc_energy_grad.argtypes = [vp, C.c_int, vp, C.c_int, dp, dp, vp, dp]
    L.mmc_phase_times.restype = st
    L.mmc_phase_times.argtypes = [vp, C.c_int64, C.c_uint64, dp, C.POINTER(C.c_int64)]
    L.mmc_angle_hist.restype = st
    L.mmc_angle_hist.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(C.c_int64), dp]
    L.mmc_trial_terms.restype = st
    L.mmc_trial_terms.argtypes = [vp, C.c_int, C.c_uint32, C.c_uint64, C.c_double, dp]
    L.mmc_set_temperature.restype = st
    L.mmc_set_temperature.argtypes = [vp, C.c_int, C.c_double, dp]
    L.mmc_minimize.restype = st
    L.mmc_minimize.argtypes = [vp, C.c_int, C.c_int64, C.c_double, C.POINTER(C.c_int64), dp, dp]
    L.mmc_sweep_serial.restype = st
    L.mmc_sweep_serial.argtypes = [vp, C.c_int64, C.c_uint64]
    L.mmc_fft_tuning.restype = st
    L.mmc_fft_tuning.argtypes = [vp, C.POINTER(C.c_int), dp]
    L.mmc_tuning.restype = st
    L.mmc_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
    L.mmc_kernel_launches.restype = C.c_int64
    L.mmc_kernel_launches.argtypes = [vp]
    L.mmc_nchains.restype = C.c_int
    L.mmc_nchains.argtypes = [vp]
    ip = C.POINTER(C.c_int)
    L.mmc_demag_kernel.restype = st
    L.mmc_demag_kernel.argtypes = [dp, ip, ip, C.c_int, C.c_int, C.c_int, C.c_int, dp]
    L.mmc_thermo.restype = st
    L.mmc_thermo.argtypes = [dp, C.c_int] + [C.c_double] * 5 + [dp] * 5
    L.mmc_ncell.restype = C.c_int64
    L.mmc_ncell.argtypes = [vp, C.c_int]
    L.mmc_checkpoint.restype = st
    L.mmc_checkpoint.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
    L.mmc_restore.restype = st
    L.mmc_restore.argtypes = [vp, vp, C.c_size_t]
    L.mmc_observables_noalloc.restype = st
    L.mmc_observables_noalloc.argtypes = [vp, C.c_int64, C.c_int, C.c_double, vp, vp, vp]
    L.mmc_checked_build.restype = C.c_int
    L.mmc_checked_build.argtypes = []
    L.mmc_check_report.restype = st
    L.mmc_check_report.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int64), C.c_int]
    L.mmc_check_total.restype = st
    L.mmc_check_total.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int)]
    L.mmc_check_site_name.restype = C.c_char_p
    L.mmc_check_site_name.argtypes = [C.c_int]
    L.mmc_status_str.restype = C.c_char_p
    L.mmc_status_str.argtypes = [st]
    L.mmc_last_error.restype = C.c_char_p
    L.mmc_last_error.argtypes = []
    _lib = L
    return L


def check(status, where):
    if status != MMC_OK:
        msg = load().mmc_last_error().decode(errors="replace")
        raise MmcError(status, where, msg)
