"""The bounds checks of the checked build (paper_2106_05593_gb300/csrc/checked.cuh),
on the host: compiled with -DMMC_CHECKED the check passes an index inside its
range through, replaces one outside (or a copy range that overruns) by the
range's start, counts every such index and records only the first; a launch
without a record is not checked; without -DMMC_CHECKED the check is the index
itself.  The normal library reports that it is not a checked build."""
import os
import shutil
import subprocess

import pytest

import paper_2106_05593_gb300 as P

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2106_05593_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "checked.cuh"
using namespace mmc;
int main() {
  MmcCheck r{};
  long long v[6];
  v[0] = MMC_CK(&r, 5, 0, 10, kCkSweepCell);
  v[1] = MMC_CK(&r, 12, 3, 10, kCkDemagField);
  v[2] = MMC_CK(&r, -1, 0, 10, kCkSweepNeighbour);
  v[3] = MMC_CKR(&r, 8, 2, 0, 10, kCkBandCopy);
  v[4] = MMC_CKR(&r, 9, 2, 0, 10, kCkBandCopy);
  v[5] = MMC_CK((MmcCheck *)nullptr, 99, 0, 10, kCkSweepCell);
  printf("%lld %lld %lld %lld %lld %lld %llu %d %lld %lld %lld %d\n", v[0], v[1], v[2], v[3], v[4], v[5],
         r.count, r.site, r.index, r.lo, r.hi, (int)kChecked);
  return 0;
}
"""


def _run(tmp_path, defines):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "ck.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / ("ck" + "".join(defines))
    subprocess.run([nvcc, *defines, "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True)
    return [int(t) for t in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]


def test_checks_in_a_checked_build(tmp_path):
    out = _run(tmp_path, ["-DMMC_CHECKED"])
    assert out[:6] == [5, 3, 0, 8, 0, 99]
    count, site, index, lo, hi, checked = out[6:]
    assert (count, index, lo, hi, checked) == (3, 12, 3, 10, 1)
    assert P.load().mmc_check_site_name(site).decode() == "demag field"


def test_checks_compile_away(tmp_path):
    out = _run(tmp_path, [])
    assert out == [5, 12, -1, 8, 9, 99, 0, 0, 0, 0, 0, 0]


def test_normal_library_is_not_checked():
    assert not P.checked_build()
    assert P.load().mmc_check_site_name(99).decode() == "?"


def test_total_is_zero_without_contexts():
    import ctypes
    n, site = ctypes.c_int64(-1), ctypes.c_int(-1)
    assert P.load().mmc_check_total(ctypes.byref(n), ctypes.byref(site)) == 0
    assert n.value == 0 and site.value == 0
