"""GPU test of mmc_observables_noalloc, the entry point for callers that cannot
allocate device memory (for example while recording a CUDA graph, or under a
framework's caching allocator).  It must give the same observables as the
context entry point mmc_observables on the same state, call after call, while
its scratch lives in a fixed array inside the library.

This file is named so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from gpu_common import lib_or_skip

pytestmark = pytest.mark.gpu

MAX_CELLS = 2097152


def call_noalloc(L, md, n, bins, hmax, out, hist, stream):
    return L.mmc_observables_noalloc(C.c_void_p(md.data_ptr()), int(n), int(bins), float(hmax),
                                     C.c_void_p(out.data_ptr()), C.c_void_p(hist.data_ptr()),
                                     C.c_void_p(stream.cuda_stream))


def test_noalloc_observables_match_the_context_entry_point():
    P = lib_or_skip()
    import torch
    L = P.load()
    mesh = (130, 77, 3)                      # 30030 cells: 30 blocks and a ragged tail
    n = int(np.prod(mesh))
    spec = W._base(mesh, (4e-9, 4e-9, 4e-9))
    g = P.MMC(spec)
    bins = 200
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    hist = torch.zeros(bins + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    for seed in (11, 12):                    # two calls in a row on different states
        m4 = W.random_state(n, seed, 0.05, 1.08)
        g.set_m(m4)
        ref = g.observables(0)
        md = torch.from_numpy(m4).cuda()
        assert call_noalloc(L, md, n, bins, 1.0, out, hist, stream) == 0, L.mmc_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        h = hist.cpu().numpy()
        assert np.array_equal(h, ref["hist"])
        assert o[0:3] == pytest.approx(ref["mean_m"], rel=1e-12, abs=1e-15)
        assert o[3] == pytest.approx(ref["mean_len"], rel=1e-12)
        assert o[4] == pytest.approx(ref["mean_len2"], rel=1e-12)
        assert o[5] == 0 and o[6] == n


def test_noalloc_counts_nonfinite_and_rejects_oversized_input():
    P = lib_or_skip()
    import torch
    L = P.load()
    n = 5000
    m4 = W.random_state(n, 3, 0.2, 0.9)
    m4[17, 1] = np.nan
    m4[4000, 2] = np.inf
    md = torch.from_numpy(m4).cuda()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    hist = torch.full((51,), 7, dtype=torch.int64, device="cuda")   # cleared by the call
    stream = torch.cuda.current_stream()
    assert call_noalloc(L, md, n, 50, 1.0, out, hist, stream) == 0
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    good = np.isfinite(m4[:, :3]).all(axis=1)
    v = m4[good, :3].astype(np.float64)
    assert o[5] == 2 and o[6] == good.sum()
    assert o[0:3] == pytest.approx(v.mean(0), rel=1e-12, abs=1e-15)
    assert int(hist.sum()) == good.sum()
    # beyond the scratch capacity: a clear error and nothing launched
    assert call_noalloc(L, md, MAX_CELLS + 1, 50, 1.0, out, hist, stream) == -1
    assert b"capacity" in L.mmc_last_error()
