"""Cases run through one build of the library by tests/test_gpu_checked.py (in a
process of its own, so that MMC_LIB_VARIANT selects the build): every kind of
sweep and demag kernel the checked build instruments, a few iterations each.
Writes the final states, the debug-pass outputs and each context's check
report to the .npz file named on the command line."""
import json
import sys

import numpy as np

import workloads as W
from paper_2106_05593_gb300 import MMC, checked_build


def _chiral(nx, ny, T=300.0):
    return W.chiral(nx, T) | {"mesh": (nx, ny, 1)}


CASES = {
    # warp-transform kernels and the fused passes (every chain padded to 1024 x 1024)
    "fused": ([_chiral(512, 512, 120.0), _chiral(301, 263, 590.0), _chiral(257, 511, 450.0)],
              dict(demag=1, fft_variant=4)),
    # interleaved 2D kernels, per-block pass; open, ragged and periodic (circular) chains
    "interleaved": ([_chiral(200, 130, 300.0), W.film256(96, 20.0) | {"mesh": (96, 80, 1)},
                     W.chiral_periodic(64, 150.0, 2)], dict(demag=1, fft_variant=1)),
    # generic kernels and the 3D pass
    "film3d": ([W._base((24, 20, 4), (3e-9, 3e-9, 2e-9), demag=True, Ms0=8e5, D0=1e-3, K1=1e5)], dict(demag=1)),
    # per-cell tables (granular chain) with demag
    "granular": ([W.granular_chain(96, 3, demag=True), W.granular_chain(64, 4, demag=True)], dict(demag=1)),
    # banded pass with bulk copies
    "band": ([W.chiral(64, 300.0), W.chiral(200, 590.0) | {"mesh": (200, 133, 1)}], dict(demag=1, sweep_tiles=1)),
    # float-float demag (generic kernels)
    "float_float": ([_chiral(200, 130, 300.0)], dict(demag=1, demag_fp64=2)),
}


def run(out_path):
    res = {"checked": int(checked_build())}
    arrays = {}
    for name, (specs, opts) in CASES.items():
        g = MMC(specs, adapt=0, stream_groups=1, **opts)
        for k, sp in enumerate(specs):
            g.set_m(W.random_state(int(np.prod(sp["mesh"])), 100 + k, 0.3, 0.9), k)
        g.sweep(3, 21)
        for k in range(len(specs)):
            arrays[f"{name}_m{k}"] = g.get_m(k)
        dec, acc = g.pass_debug(0, 1, 5, 22, 20.0)
        arrays[f"{name}_dec"] = dec
        arrays[f"{name}_acc"] = acc
        res[name] = g.check_report()
    np.savez(out_path, **arrays)
    print(json.dumps(res))


if __name__ == "__main__":
    run(sys.argv[1])
