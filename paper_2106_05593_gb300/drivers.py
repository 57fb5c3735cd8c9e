"""Host drivers on top of the MMC library.

switching_trace() / crossing_probability(): the switching comparison of
App. B between the parallel form (demag field once per iteration, Eq. 14) and
the serial form (field updated after every accepted move).

hysteresis(): the field-loop protocol of Sec. III.  For every field value the
chains run chunks of iterations (2000 in the paper), each chunk averaging the
magnetization; a field step is accepted once at least two chunks have run and the
last two chunk averages of m along the field direction differ by less than the
threshold (0.01 in the paper), which spends few iterations where the loop changes
slowly and many at switching events.  All work runs in the library; this module
only sequences calls and reads back the chunk averages.
"""
from __future__ import annotations

import numpy as np


def chunk_converged(history, threshold, min_chunks=2):
    """True once >= min_chunks chunk averages exist and the last two differ by < threshold."""
    return len(history) >= min_chunks and abs(history[-1] - history[-2]) < threshold


def hysteresis(engine, fields, seed, chunk=2000, threshold=0.01, min_chunks=2, max_chunks=50,
               sample_every=10, chains=None):
    """Run a field loop on every chain of `engine` (an MMC context).

    fields: sequence of applied fields (tesla, 3-vectors), applied to all chains.
    Returns a dict with, per field, the accepted chunk average of m along the
    field direction for each chain, the chunks used, and the iterations spent.
    """
    chains = list(range(engine.nchains)) if chains is None else list(chains)
    out = {"field": [], "m_par": [], "chunks": [], "iterations": 0}
    for B in fields:
        B = np.asarray(B, dtype=np.float64)
        nrm = np.linalg.norm(B)
        bhat = B / nrm if nrm > 0 else np.array([1.0, 0.0, 0.0])
        engine.set_field(B, -1)
        for k in chains:
            engine.observables(k, reset=True)          # clear the snapshot accumulators
        hist = {k: [] for k in chains}
        done = {k: False for k in chains}
        used = 0
        while not all(done.values()) and used < max_chunks:
            engine.sweep_sampled(chunk, seed, sample_every)
            used += 1
            out["iterations"] += chunk
            for k in chains:
                ob = engine.observables(k, reset=True)
                if not done[k]:
                    hist[k].append(float(np.dot(ob["mean_m"], bhat)))
                    done[k] = chunk_converged(hist[k], threshold, min_chunks)
        out["field"].append(B.tolist())
        out["m_par"].append([hist[k][-1] for k in chains])
        out["chunks"].append([len(hist[k]) for k in chains])
    return out


def switching_trace(engine, n_iter, seed, every=10, serial=False, axis=(1.0, 0.0, 0.0)):
    """Run n_iter iterations on every chain of `engine` (parallel form, or the
    serial exact-demag form when serial=True) and record, after every `every`
    iterations, each chain's mean m along `axis` (App. B, Fig. 12a).
    Returns (iterations, trace) with trace[sample, chain]."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    step = engine.sweep_serial if serial else engine.sweep
    for k in range(engine.nchains):
        engine.observables(k, reset=True)              # observables of the current state below
    its, rows = [], []
    done = 0
    while done < n_iter:
        k = min(every, n_iter - done)
        step(k, seed)
        done += k
        its.append(done)
        rows.append([float(np.dot(engine.observables(c)["mean_m"], a)) for c in range(engine.nchains)])
    return np.asarray(its), np.asarray(rows)


def crossing_probability(trace):
    """Fraction of chains whose m along the axis has become positive at or
    before each sample (App. B, Fig. 12b)."""
    crossed = np.maximum.accumulate(np.asarray(trace) > 0.0, axis=0)
    return crossed.mean(axis=1)


def angular_histogram(engine, chain, nsnap, every, seed, bins=100, lo=0.0, hi=np.pi):
    """The transverse check of Sec. II (Fig. 1d-f): after every `every`
    iterations the polar angle of each cell to the configuration's mean
    direction is histogrammed; returns the bin centres and the histogram
    averaged over nsnap configurations, normalized to unit area."""
    acc = np.zeros(bins)
    for _ in range(nsnap):
        engine.sweep(every, seed)
        h, _ = engine.angle_hist(chain, bins, lo, hi)
        acc += h[:bins]
    width = (hi - lo) / bins
    centres = lo + (np.arange(bins) + 0.5) * width
    total = acc.sum()
    return centres, (acc / (total * width) if total > 0 else acc)


TERM_NAMES = ("exchange", "dmi", "anisotropy", "zeeman", "longitudinal", "demag")


def trial_term_averages(engine, chain, nsnap, every, seed):
    """The per-term free-energy changes of the trial moves (App. B, Fig. 11):
    after every `every` iterations the mean |dF| / kT of each term over the
    trial moves of all cells of the chain (the moves of the next iteration, at
    the chain's current cone angle) is taken; returns a dict of the averages
    over nsnap configurations."""
    acc = np.zeros(6)
    for _ in range(nsnap):
        engine.sweep(every, seed)
        sweep = int(engine.observables(chain)["sweeps"])
        acc += engine.trial_terms(chain, sweep, seed, -1.0)
    acc /= max(nsnap, 1)
    return dict(zip(TERM_NAMES, acc))
