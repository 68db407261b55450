"""Autotuner for the row-bin thresholds (hs_set_tuning).

The tables of the accumulators have fixed capacities; the thresholds decide
which rows take the smaller tiers (smaller tables, more rows in flight per SM)
and which rows the bitmap kernel serves.  The best setting depends on the
workload's mix of row sizes, so it is measured: one coordinate-descent sweep
over each threshold's candidate values, each setting timed with CUDA events
(median of `trials` runs after one warm-up) on the caller's workload.
Results never depend on the thresholds, only the time does.
"""
from __future__ import annotations

import statistics

from . import hspgemm as h

# candidate values per threshold (the first ones switch a tier off)
CANDIDATES = {
    "warp_s_max": (32, 64, 128),
    "mid_s_max": (0, 512, 768, 1024),
    "large_s_max": (2048, 3072, 4096),
    "sym_mid_s_max": (512, 768, 1024),
    "sym_heavy_from": (4096, 6144, 0),
    "sort_pct": (101, 25, 50, 75, 90),
    "sort_max": (256, 512, 1024),
}


def time_ms(run, trials: int, stream=None) -> float:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    run()
    ts = []
    for _ in range(trials):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        run()
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune(run, trials: int = 3, candidates: dict | None = None, stream=None):
    """Pick the thresholds that make `run()` fastest; leaves them set.

    Returns (best, log): best is the chosen tuning dict, log a list of
    (tuning, ms) for every setting timed (the first is the defaults)."""
    cands = CANDIDATES if candidates is None else candidates
    h.set_tuning(None)
    best = h.get_tuning()
    best_ms = time_ms(run, trials, stream)
    log = [(dict(best), best_ms)]
    for knob, values in cands.items():
        start = best[knob]  # timed already, with the same other knobs: best_ms
        for v in values:
            if v == start:
                continue
            trial = dict(best, **{knob: v})
            h.set_tuning(trial)
            ms = time_ms(run, trials, stream)
            log.append((dict(trial), ms))
            if ms < best_ms:
                best, best_ms = dict(trial), ms
        h.set_tuning(best)
    return best, log
