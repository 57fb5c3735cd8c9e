import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical test")


def pytest_terminal_summary(terminalreporter):
    """Totals of the one-pass accept/reject comparisons of the session: flips are
    allowed only inside the 1e-6 kT band (Eq. 5 decision values)."""
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
