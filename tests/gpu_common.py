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


def oracle_pass(spec, m4, color, sweep, chain, seed, theta, H=None):
    """Oracle sublattice pass on an FP32 state given as (n, 4)."""
    o = O.Oracle(spec)
    m = m4[:, :3].astype(np.float64)
    if spec.get("demag") and H is None:
        H = o.demag_field(m, "fft" if o.n > 1024 else "direct")
    m1, acc, dec, band = o.sweep_pass(m, H, color, sweep, chain, seed, theta)
    return m1, acc, dec, band


def compare_pass(dec_g, acc_g, dec_o, acc_o, band_o, strict=1e-6, rel=2e-6, absolute=5e-5):
    """Accept bits must agree wherever the oracle's decision value is farther from
    0 than the FP32 error bound of the GPU's decision value.  Returns stats."""
    sel = acc_o >= 0
    assert np.array_equal(acc_g < 0, acc_o < 0), "colour masks differ"
    d_o = dec_o[sel]
    d_g = dec_g[sel].astype(np.float64)
    b = band_o[sel]
    bound = absolute + rel * b
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
