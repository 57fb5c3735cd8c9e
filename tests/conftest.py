import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical test")


def _checked_total():
    """(count, site name) of the out-of-range indices the checked build met in
    the contexts destroyed so far; None when the normal build is loaded."""
    if os.environ.get("MMC_LIB_VARIANT") != "checked":
        return None
    import ctypes
    import gc

    import paper_2106_05593_gb300 as P
    gc.collect()
    n, site = ctypes.c_int64(0), ctypes.c_int(0)
    P.load().mmc_check_total(ctypes.byref(n), ctypes.byref(site))
    return int(n.value), P.load().mmc_check_site_name(site.value).decode()


def pytest_sessionfinish(session, exitstatus):
    """Run on the checked build (MMC_LIB_VARIANT=checked), the session fails if
    any kernel met an index outside its buffer region."""
    r = _checked_total()
    if r is not None and r[0] > 0:
        session.exitstatus = 1


def pytest_terminal_summary(terminalreporter):
    """Totals of the one-pass accept/reject comparisons of the session: flips are
    allowed only inside the 1e-6 kT band (Eq. 5 decision values); on the checked
    build, the out-of-range indices met."""
    r = _checked_total()
    if r is not None:
        terminalreporter.write_line(f"checked build: {r[0]} out-of-range indices (first at: {r[1]})")
    try:
        import gpu_common
    except ImportError:
        return
    st = gpu_common.PASS_STATS
    if not st:
        return
    tot = {k: sum(s[k] for s in st) for k in ("n", "mismatch", "mismatch_strict", "mismatch_between",
                                              "mismatch_outside_bound")}
    worst = max(s["max_err_over_bound"] for s in st)
    terminalreporter.write_line(
        f"one-pass comparisons: {len(st)} passes, {tot['n']} cells, flips {tot['mismatch']} "
        f"(inside 1e-6 kT: {tot['mismatch_strict']}, between 1e-6 kT and the FP32 bound: "
        f"{tot['mismatch_between']}, outside: {tot['mismatch_outside_bound']}); "
        f"largest decision error / bound {worst:.3f}")
