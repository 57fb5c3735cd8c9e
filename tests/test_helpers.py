"""CPU checks of the GPU tests' comparison helpers (no GPU): the histogram rule
accepts an FP32 binning that differs from the FP64 one only at bin edges and
rejects a cell moved anywhere else."""
import numpy as np
import pytest

from gpu_common import compare_hist


def _f32_hist(m4, bins, hmax):
    """An independent FP32 binning (numpy float32 arithmetic) standing in for a
    GPU histogram."""
    v = m4[:, :3].astype(np.float32)
    r = np.sqrt((v * v).sum(axis=1, dtype=np.float32))
    t = r * np.float32(bins / hmax)
    b = np.minimum(np.floor(t).astype(np.int64), bins)
    return np.bincount(b, minlength=bins + 1)


def test_compare_hist_accepts_edge_cells_and_rejects_moves():
    rng = np.random.default_rng(5)
    n, bins = 20000, 200
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    L = rng.uniform(0.2, 1.05, n)
    L[:50] = (rng.integers(1, bins, 50)) / bins     # exactly on bin edges in FP64
    m4 = np.zeros((n, 4), np.float32)
    m4[:, :3] = (d * L[:, None]).astype(np.float32)
    h = _f32_hist(m4, bins, 1.0)
    namb = compare_hist(h, m4, bins, 1.0)
    assert namb >= 1
    bad = h.copy()
    k = int(np.argmax(bad[10:150])) + 10
    bad[k] -= 1
    bad[k + 2] += 1
    with pytest.raises(AssertionError):
        compare_hist(bad, m4, bins, 1.0)


def test_granular_sizes_cover_even_sides():
    """The granular batch's square sides are even values of 64..1024 drawn
    uniformly: not only multiples of 32 (the kernels take any even side)."""
    import workloads as W
    s = np.array(W.granular_sizes(2000, seed=3))
    assert s.min() >= 64 and s.max() <= 1024 and (s % 2 == 0).all()
    assert (s % 32 != 0).mean() > 0.9
    assert abs(s.mean() - 544.0) < 15.0
    assert W.granular_sizes() == W.granular_sizes()          # seeded
