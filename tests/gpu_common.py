"""Helpers shared by the GPU parity tests: building/loading the library and
running the oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O


def lib_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_05593_gb300 import build
    build.build()
    import paper_2106_05593_gb300 as P
    P.load()
    return P


def oracle_pass(spec, m4, color, sweep, chain, seed, theta, H=None, o=None):
    """Oracle sublattice pass on an FP32 state given as (n, 4) (o: an oracle of
    spec to reuse, or None)."""
    o = O.Oracle(spec) if o is None else o
    m = m4[:, :3].astype(np.float64)
    if spec.get("demag") and H is None:
        H = o.demag_field(m, "fft" if o.n > 1024 else "direct")
    m1, acc, dec, band = o.sweep_pass(m, H, color, sweep, chain, seed, theta)
    return m1, acc, dec, band


def exchange_weight_sum(spec):
    """Sum over a cell's bonds of the exchange weights V A0 / (h_a^2 kT) (kT units,
    at the lowest temperature of the spec)."""
    h = spec["h"]
    V = h[0] * h[1] * h[2]
    T = float(np.min(spec["T"]))
    axes = 3 if spec["mesh"][2] > 1 else 2
    return sum(2.0 * V * spec.get("A0", 0.0) / (h[a] ** 2 * 1.380649e-23 * T) for a in range(axes))


def compare_pass(dec_g, acc_g, dec_o, acc_o, band_o, strict=1e-6, rel=2e-6, absolute=5e-5, wsum=0.0):
    """Accept bits must agree wherever the oracle's decision value is at least
    `strict` (1e-6 kT) from 0, and decision values within the FP32 error bound of
    the GPU's decision value.  Returns stats.

    The bound is absolute + rel * band + 1e-6 * wsum.  The last term is the
    rounding of the FP32 proposal: the GPU's m' differs from the oracle's FP64 m'
    by a few FP32 ulps (|dm'| <= 4 * 2^-24 |m|), and the exchange change
    sum_b w_b (|m' - m_b|^2 - |m - m_b|^2) moves by 2 sum_b w_b |m' - m_b| |dm'|
    <= 2 * wsum * 2.2 * 2.4e-7 ~ 1e-6 * wsum for |m| <= 1.1, independently of the
    size of the exchange change itself (wsum = exchange_weight_sum(spec))."""
    sel = acc_o >= 0
    assert np.array_equal(acc_g < 0, acc_o < 0), "colour masks differ"
    d_o = dec_o[sel]
    d_g = dec_g[sel].astype(np.float64)
    b = band_o[sel]
    bound = absolute + rel * b + 1e-6 * wsum
    err = np.abs(d_g - d_o)
    mism = acc_g[sel] != acc_o[sel]
    stats = {
        "n": int(sel.sum()), "max_err": float(err.max(initial=0.0)),
        "max_err_over_bound": float((err / bound).max(initial=0.0)),
        "mismatch": int(mism.sum()),
        "mismatch_strict": int((mism & (np.abs(d_o) < strict)).sum()),
        "mismatch_outside_bound": int((mism & (np.abs(d_o) >= bound)).sum()),
    }
    # flips with strict <= |d| < bound: allowed by the FP32 error bound, but not by
    # the 1e-6 kT band of the accept/reject comparison, so none may occur
    stats["mismatch_between"] = stats["mismatch"] - stats["mismatch_strict"] - stats["mismatch_outside_bound"]
    PASS_STATS.append(stats)
    assert stats["max_err_over_bound"] <= 1.0, stats
    assert stats["mismatch_outside_bound"] == 0, stats
    assert stats["mismatch_between"] == 0, stats
    return stats


# every compare_pass of the session (summed in the terminal summary, conftest.py)
PASS_STATS = []


def compare_hist(h_gpu, m4, bins=200, hmax=1.0, rel=1e-6):
    """The GPU's |m| histogram of the FP32 state m4 against the oracle's FP64
    binning.  A cell whose FP64 bin position t = |m| bins / hmax lies within
    FP32 rounding of a bin edge (|t - round(t)| <= rel * max(t, 1); FP32 forms
    |m| with a relative error of a few 2^-24) may fall on either side of that
    edge; every other cell must be in the oracle's bin.  Returns the number of
    such edge cells."""
    import oracle as O
    v = np.asarray(m4)[:, :3].astype(np.float64)
    t = np.linalg.norm(v, axis=1) / hmax * bins
    e = np.rint(t)
    amb = (np.abs(t - e) <= rel * np.maximum(t, 1.0)) & (e >= 1) & (e <= bins)
    h_sure = O.hist(v[~amb], bins, hmax)
    D = np.asarray(h_gpu, dtype=np.int64) - h_sure
    assert D.sum() == int(amb.sum()) and (D >= 0).all(), (D[D != 0], int(amb.sum()))
    # a_e cells at edge e (between bins e - 1 and e): x_e of them go up, the rest
    # down; D[b] = x_b + (a_{b+1} - x_{b+1}) must be solvable with 0 <= x <= a
    a = np.bincount(e[amb].astype(np.int64), minlength=bins + 2)
    carry = 0                               # x_b: cells of edge b that went up into bin b
    for b in range(bins + 1):
        down = D[b] - carry                 # cells of edge b + 1 that went down into bin b
        nxt = a[b + 1] if b + 1 <= bins else 0
        assert 0 <= down <= nxt, ("histogram differs outside the FP32 edge band", b, D[b], carry, nxt)
        carry = nxt - down
    assert carry == 0
    return int(amb.sum())


def welch_z(a, b):
    """z = (mean a - mean b) / SE of the difference, SE from the spread of the
    independent chains of each side (a, b: one value per chain)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    se = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
    d = a.mean() - b.mean()
    if se == 0.0:
        return 0.0 if d == 0.0 else np.inf
    return float(d / se)


def hist_cdf(h, edges):
    """Fractions of a histogram's counts in the bins below each edge index."""
    h = np.asarray(h, dtype=np.float64)
    c = np.cumsum(h) / h.sum()
    return np.array([c[e - 1] for e in edges])
