"""The bench's kernel-source hash ignores comments but not code, and the
recorded ncu traffic is found only for the hash it was taken on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench
    finally:
        sys.argv = argv
    return bench


def test_hash_ignores_comments_only():
    b = _bench()
    src = {f: open(os.path.join(ROOT, "paper_2106_05593_gb300", "csrc", f)).read() for f in b.KERNEL_SOURCES}
    base = b.kernel_source_hash(lambda f: src[f])
    assert base == b.kernel_source_hash()
    commented = dict(src)
    commented["k_sweep.cu"] = "// a new comment\n" + src["k_sweep.cu"].replace("{", "{  /* x */", 1)
    assert b.kernel_source_hash(lambda f: commented[f]) == base
    changed = dict(src)
    changed["k_sweep.cu"] = src["k_sweep.cu"].replace("kSweepCells = 2", "kSweepCells = 4", 1)
    assert changed["k_sweep.cu"] != src["k_sweep.cu"]
    assert b.kernel_source_hash(lambda f: changed[f]) != base


def test_recorded_traffic_keyed_by_hash():
    b = _bench()
    rows = [ln.split() for ln in open(os.path.join(ROOT, "profiles", "dram_traffic_per_launch.txt"))
            if ln.strip() and not ln.startswith("#")]
    kernel, workload, h, value = rows[0][:4]
    assert b.recorded_traffic(kernel, workload, h) == float(value)
    assert b.recorded_traffic(kernel, workload, "0" * 16) is None
