"""The bounds-checked build on the GPU (libmmc_checked.so, -DMMC_CHECKED): every
sweep and demag kernel it instruments (warp-transform and fused kernels,
interleaved and generic transforms, the one-cell-thick, 3D and banded passes,
per-cell tables, float-float demag, the debug pass) runs a few iterations of
uneven, ragged, periodic and 3D chains without a single index out of its
range, and ends in the states the normal build reaches (to FP32 rounding:
the checks change how the compiler schedules the arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")


def _run_cases(out, variant):
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([ROOT, TESTS, os.environ.get("PYTHONPATH", "")]))
    if variant:
        env["MMC_LIB_VARIANT"] = variant
    else:
        env.pop("MMC_LIB_VARIANT", None)
    r = subprocess.run([sys.executable, os.path.join(TESTS, "checked_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(out)


def test_checked_build_finds_no_bad_index(tmp_path):
    lib_or_skip()
    subprocess.run([sys.executable, "-c", "from paper_2106_05593_gb300 import build; build.build(checked=True)"],
                   cwd=ROOT, check=True, timeout=1800)
    rep_c, arr_c = _run_cases(tmp_path / "checked.npz", "checked")
    rep_n, arr_n = _run_cases(tmp_path / "normal.npz", None)
    assert rep_c["checked"] == 1 and rep_n["checked"] == 0
    for name, r in rep_c.items():
        if name == "checked":
            continue
        print(name, r)
        assert r["count"] == 0, (name, r)
        assert rep_n[name]["count"] == 0
    for key in arr_n.files:
        a, b = arr_c[key], arr_n[key]
        if key.endswith("_acc"):
            assert int((a != b).sum()) <= 2, key
        elif key.endswith("_dec"):
            assert np.abs(a.astype(np.float64) - b).max() < 1e-3, key
        else:
            d = np.abs(a[:, :3].astype(np.float64) - b[:, :3]).max(axis=1)
            nd = int((d > 1e-5).sum())
            print(key, "differing cells", nd, "max |dm| elsewhere %.2e" % d[d <= 1e-5].max(initial=0.0))
            assert nd <= 3 and d[d <= 1e-5].max(initial=0.0) < 1e-6, key
