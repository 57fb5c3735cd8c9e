"""Parity at the benchmark's full sizes, in its launch configuration: the
16-chain chiral batch (512 x 512 cells per chain, demag on, FP32 demag with the
FFT variant picked at create) and the probe film (8192 x 8192 cells, one chain).
One sublattice pass of selected chains is compared element by element with the
oracle's pass on the same state (for the probe on a sampled block of rows,
which the oracle can compute one by one); the rest of the batch is checked to be
untouched by the diagnostic pass."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import compare_pass, exchange_weight_sum, lib_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return lib_or_skip()


@pytest.mark.parametrize("chain", [0, 9, 15])
def test_chiral_batch_full_size_pass(P, chain):
    specs = W.chiral512_batch()
    g = P.MMC(specs, demag=1)
    g.init_random(7)
    g.sweep(3, 7)                                   # a non-trivial state of every chain
    m4 = g.get_m(chain)
    other = g.get_m((chain + 1) % 16)
    o = O.Oracle(specs[chain])
    m = m4[:, :3].astype(np.float64)
    H = o.demag_field(m, "fft")
    for color in (0, 1):
        g.set_m(m4, chain)
        dec_g, acc_g = g.pass_debug(chain, color, 11, 99, 20.0)
        _, acc_o, dec_o, band_o = o.sweep_pass(m, H, color, 11, chain, 99, 20.0)
        st = compare_pass(dec_g, acc_g, dec_o, acc_o, band_o, wsum=exchange_weight_sum(specs[chain]))
        print("chiral batch chain %d colour %d: %s" % (chain, color, st))
    assert np.array_equal(g.get_m((chain + 1) % 16), other)


@pytest.mark.parametrize("color", [0, 1])
def test_probe_full_size_pass_on_sampled_rows(P, color):
    """The 8192 x 8192 probe film (one chain, 67 M cells): one pass of the whole
    film on the GPU; the oracle computes a band of 64 rows as a window of the
    lattice (its cells carry their global indices into the random numbers), and
    the band's interior rows, whose neighbours all lie in the band, must agree
    element by element."""
    nx = 8192
    spec = W.probe(nx)
    g = P.MMC(spec)
    g.init_random(3)
    g.sweep(2, 3)
    m4 = g.get_m()
    dec_g, acc_g = g.pass_debug(0, color, 5, 21, 30.0)
    for r0 in (0, 4000, nx - 64):                   # an edge band, a middle band, the far edge
        nr = 64
        band = m4.reshape(nx, nx, 4)[r0:r0 + nr].reshape(-1, 4)
        sub = dict(spec, mesh=(nx, nr, 1), cell_base=r0 * nx)
        o = O.Oracle(sub)
        _, acc_o, dec_o, band_o = o.sweep_pass(band[:, :3].astype(np.float64), None, color if r0 % 2 == 0 else 1 - color,
                                               5, 0, 21, 30.0)
        lo = 0 if r0 == 0 else 1                    # film edge rows are real edges
        hi = nr if r0 + nr == nx else nr - 1
        sl_o = slice(lo * nx, hi * nx)
        sl_g = slice((r0 + lo) * nx, (r0 + hi) * nx)
        st = compare_pass(dec_g[sl_g], acc_g[sl_g], dec_o[sl_o], acc_o[sl_o], band_o[sl_o],
                          wsum=exchange_weight_sum(spec))
        print("probe 8192^2 colour %d rows %d..%d: %s" % (color, r0 + lo, r0 + hi, st))


def _differing(mg, mo, tol=1e-5):
    d = np.abs(mg - mo).max(axis=1)
    return int((d > tol).sum()), float(d[d <= tol].max(initial=0.0))


def test_chiral_batch_full_size_iterations(P):
    """The benchmarked path itself (the production pass kernel, the create-time
    FFT variant, chain groups on concurrent streams) over three whole
    iterations of the 16-chain batch: chains 0, 9 and 15 end equal to the
    oracle's run from the same state to FP32 rounding, except the few cells a
    decision inside the FP32 bound can change (a flipped cell and, later, its
    neighbours)."""
    specs = W.chiral512_batch()
    g = P.MMC(specs, demag=1)
    g.init_random(7)
    start = {k: g.get_m(k) for k in (0, 9, 15)}
    g.sweep(3, 7)
    for k, m4 in start.items():
        o = O.Oracle(specs[k])
        st = O.new_state(seed=7, chain=k, theta_deg=30.0, adapt=True, demag_mode=1)
        mo, _, _ = o.run(m4[:, :3].astype(np.float64), 3, st)
        ndiff, agree = _differing(g.get_m(k)[:, :3].astype(np.float64), mo)
        print("chiral batch chain %d, 3 iterations: differing cells %d, max |dm| elsewhere %.2e" % (k, ndiff, agree))
        assert agree < 1e-5 and ndiff <= 8


def test_chiral_batch_full_size_graphs_equal_eager(P):
    """A 100-iteration block of the full batch replayed as a CUDA graph (the
    benchmark's launch form) equals the same iterations launched eagerly, bit
    for bit, for every chain."""
    specs = W.chiral512_batch()
    a = P.MMC(specs, demag=1)
    variant = a.fft_tuning()[0]
    b = P.MMC(specs, demag=1, use_graphs=0, fft_variant=variant)
    for g in (a, b):
        g.init_random(11)
        g.sweep(100, 11)
    for k in range(16):
        assert np.array_equal(a.get_m(k), b.get_m(k)), k
    assert [a.observables(k)["theta_deg"] for k in range(16)] == [b.observables(k)["theta_deg"] for k in range(16)]


def test_probe_full_size_iterations_on_windows(P):
    """Two whole iterations of the 8192 x 8192 probe film through mmc_sweep (the
    production kernel) against the oracle's run of three 64-row windows of the
    same state; rows within four of a window's cut see stale neighbours in the
    oracle (four passes) and are left out."""
    nx = 8192
    spec = W.probe(nx)
    g = P.MMC(spec, adapt=0)
    g.init_random(5)
    g.sweep(2, 5)                                   # a non-trivial start
    m0 = g.get_m().reshape(nx, nx, 4)
    g.sweep(2, 9)
    m1 = g.get_m().reshape(nx, nx, 4)
    for r0 in (0, 4000, nx - 64):                   # even: window colours equal global colours
        nr = 64
        sub = dict(spec, mesh=(nx, nr, 1), cell_base=r0 * nx)
        o = O.Oracle(sub)
        st = O.new_state(seed=9, chain=0, theta_deg=30.0, adapt=False, demag_mode=0, sweep=2)
        mo, _, _ = o.run(m0[r0:r0 + nr].reshape(-1, 4)[:, :3].astype(np.float64), 2, st)
        lo = 0 if r0 == 0 else 4
        hi = nr if r0 + nr == nx else nr - 4
        mg = m1[r0 + lo:r0 + hi].reshape(-1, 4)[:, :3].astype(np.float64)
        ndiff, agree = _differing(mg, mo.reshape(nr, nx, 3)[lo:hi].reshape(-1, 3))
        print("probe rows %d..%d, 2 iterations: differing cells %d, max |dm| elsewhere %.2e"
              % (r0 + lo, r0 + hi, ndiff, agree))
        assert agree < 1e-5 and ndiff <= 8
