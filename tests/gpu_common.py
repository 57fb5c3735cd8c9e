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
    """Accept bits must agree wherever the oracle's decision value is farther from
    0 than the FP32 error bound of the GPU's decision value.  Returns stats.

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
    assert stats["max_err_over_bound"] <= 1.0, stats
    assert stats["mismatch_outside_bound"] == 0, stats
    return stats
