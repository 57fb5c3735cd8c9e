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


def test_cpu_sample_of_the_workloads():
    """The oracle's CPU sample: a corner block of large chains (per-cell arrays
    cut alike) and one periodic image per side for periodic demag kernels."""
    import numpy as np
    import workloads as W
    b = _bench()
    spec = W._base((1024, 600, 2), (2e-9, 2e-9, 2e-9), Ms0=np.arange(1024 * 600 * 2, dtype=np.float64))
    out, what = b.crop_spec(spec)
    assert out["mesh"] == (512, 512, 2) and what.startswith("corner block")
    ms = out["Ms0"].reshape(2, 512, 512)
    assert ms[1, 3, 5] == 1024 * 600 + 3 * 1024 + 5
    per = W.chiral_periodic(512, 300.0, 10)
    out, what = b.crop_spec(per)
    assert out["demag_images"] == b.CPU_SAMPLE_IMAGES and "image" in what and out["mesh"] == per["mesh"]
    small = W.permalloy32()
    out, what = b.crop_spec(small)
    assert out is small and what == "chain 0"


def test_spectrum_bytes_follow_the_transform():
    import workloads as W
    b = _bench()
    assert b.spectrum_bytes_per_cell([W.chiral(512, 300.0)]) == 24.0
    assert b.spectrum_bytes_per_cell([W.chiral_periodic(512, 300.0, 4)]) == 12.0
    assert b.spectrum_bytes_per_cell([W.chiral_periodic(500, 300.0, 4)]) == 24.0     # not a power of two
    assert b.algorithmic_bytes("demag_cols", True, False, 12.0) == 24.0
