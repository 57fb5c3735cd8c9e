"""GPU tests of the create-time autotuner of the batched form: it times the FP32
FFT variants and 1, 2, 3 chain groups on the batch, keeps the fastest, and
records the picks in the tuning cache, so that a second create of the same
problem reads them instead of timing and runs the same kernels (bit-identical
chains); other problems and a disabled cache time afresh."""
import os

import numpy as np
import pytest

import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


def _batch(n=64):
    return [W.chiral(n, 100.0 + 120.0 * k) for k in range(4)]


def test_tuner_times_then_reads_the_cache(P, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("MMC_TUNE_CACHE", str(cache))
    a = P.MMC(_batch(), demag=1)
    ta = a.tuning()
    assert not ta["from_cache"]
    assert ta["stream_groups"] in (1, 2, 3) and ta["fft_variant"] in (1, 2, 3)
    assert all(t > 0 for t in ta["groups_ms"][:3]) and ta["fft_ms"][0] > 0
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:] == [str(ta["fft_variant"]), str(ta["stream_groups"])]
    b = P.MMC(_batch(), demag=1)
    tb = b.tuning()
    assert tb["from_cache"] and tb["fft_variant"] == ta["fft_variant"] and tb["stream_groups"] == ta["stream_groups"]
    for g in (a, b):
        g.init_random(3)
        g.sweep(150, 3)
    for k in range(4):
        assert np.array_equal(a.get_m(k), b.get_m(k)), k
    # another problem is timed and gets its own line; a garbled line is ignored
    with open(cache, "a") as f:
        f.write("garbage line\n")
    c = P.MMC(_batch(48), demag=1)
    assert not c.tuning()["from_cache"]
    assert len(cache.read_text().splitlines()) == 3


def test_tuner_without_cache(P, tmp_path, monkeypatch):
    monkeypatch.setenv("MMC_TUNE_CACHE", "off")
    a = P.MMC(_batch(), demag=1)
    b = P.MMC(_batch(), demag=1)
    assert not a.tuning()["from_cache"] and not b.tuning()["from_cache"]
    assert not any(os.scandir(tmp_path))
    # explicit choices are not tuned
    c = P.MMC(_batch(), demag=1, fft_variant=1, stream_groups=2)
    t = c.tuning()
    assert t["fft_variant"] == 1 and t["stream_groups"] == 2 and t["groups_ms"] == (0.0, 0.0, 0.0)
