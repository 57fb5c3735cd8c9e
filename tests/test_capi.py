"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/mmc.h declares.  No compute call is made."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mmc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mmc_[a-z0-9_]+)\s*\(", txt)))


def test_header_lists_the_documented_entry_points():
    names = declared_functions()
    from paper_2106_05593_gb300 import EXPORTS
    assert sorted(EXPORTS) == names


def test_library_builds_loads_and_exports_every_symbol():
    pytest.importorskip("ctypes")
    from paper_2106_05593_gb300 import build, load
    try:
        build.build()
    except RuntimeError as e:   # no CUDA toolkit on this machine
        pytest.skip(str(e))
    L = load()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_noalloc_rejects_misaligned_pointers_before_any_launch():
    """mmc_observables_noalloc checks the alignment of its device pointers on
    the host and returns MMC_ERR_ARG without touching them or the GPU (the
    pointer values here are never dereferenced)."""
    import ctypes as C
    from paper_2106_05593_gb300 import build, load
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    L = load()
    f = L.mmc_observables_noalloc
    base = 1 << 20
    for m, out, hist in ((base + 4, base, base), (base + 8, base, base), (base, base + 4, base),
                         (base, base, base + 2)):
        rc = f(C.c_void_p(m), 100, 50, C.c_double(1.0), C.c_void_p(out), C.c_void_p(hist), None)
        assert rc == -1, (m, out, hist, rc)
        assert b"aligned" in L.mmc_last_error()
