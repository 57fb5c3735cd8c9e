"""GB300 (sm_103a) implementation of the parallel micromagnetic Monte Carlo method
(Lepadatu, arXiv:2106.05593): red-black Metropolis sweeps with cone + length
moves, FFT demag convolution, observables and energies, behind the C ABI of
include/mmc.h.  This package is the thin Python binding of that library.
"""
from ._lib import EXPORTS, MmcError, load  # noqa: F401
from .mmc import MMC, checked_build, default_options, demag_kernel, thermo  # noqa: F401

__all__ = ["MMC", "checked_build", "default_options", "demag_kernel", "thermo", "MmcError", "load", "EXPORTS"]
