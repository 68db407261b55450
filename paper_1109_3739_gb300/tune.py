"""Autotuner for the row-bin thresholds (hs_set_tuning).

The tables of the accumulators have fixed capacities; the thresholds decide
which rows take the smaller tiers (smaller tables, more rows in flight per SM),
which rows sort their products instead of hashing them (sort_max, sort_pct)
and which rows the bitmap kernel serves.  The best setting depends on the
workload's mix of row sizes, so it is measured: one coordinate-descent sweep
over each threshold's candidate values, each setting timed with CUDA events
(median of `trials` runs after one warm-up) on the caller's workload.
tune_cached() keeps the choice in a JSON file keyed by the GPU, the
semiring, the value type and the shape of the work (work_shape), so a
workload of the same shape is tuned once.  Results never depend on the
thresholds, only the time does.
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
    "sym_heavy_from": (0, 6144, 8192),
    "sort_pct": (101, 25, 50, 75, 90),
    "sort_max": (256, 512, 1024),
    "spa_max": (0, 2048),
    "heavy_part_kb": (16, 32),
    "num_heavy_from": (0, 4096, 8192),
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


# ------------------------------------------------------------------ cache
# A tuning is chosen once per (GPU, semiring, value type, shape of the work):
# the work's shape is the share of the product's multiplications that falls
# in each power-of-two band of row products, rounded to 5 %, together with
# the output/product ratio rounded to a tenth.  Workloads that agree on these
# take the same bins, so the cached thresholds fit them without timing again.
FLOP_BANDS = (32, 128, 256, 512, 1024, 4096, 8192, 16384, 1 << 62)


def work_shape(row_flops, nnz_c: int | None = None) -> dict:
    """The key's workload part from the products per row (any array-like of
    non-negative integers) and, if known, nnz(C)."""
    import numpy as np
    f = np.asarray(row_flops, dtype=np.int64)
    total = int(f.sum())
    shares = []
    lo = 0
    for hi in FLOP_BANDS:
        part = int(f[(f > lo) & (f <= hi)].sum())
        shares.append(round(20 * part / total) * 5 if total else 0)
        lo = hi
    shape = {"bands": shares}
    if nnz_c is not None and total:
        shape["c_per_flop"] = round(10 * nnz_c / total) / 10
    return shape


def cache_key(device_name: str, semiring: str, dtype: str, shape: dict) -> str:
    import json
    return json.dumps({"gpu": device_name, "semiring": semiring, "dtype": dtype, **shape}, sort_keys=True)


def default_cache_path() -> str:
    import os
    base = os.environ.get("HS_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "hspgemm", "tuning.json")


def _load(path: str) -> dict:
    import json
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def tune_cached(run, key: str, trials: int = 3, candidates: dict | None = None, stream=None,
                path: str | None = None):
    """tune() once per key: a cached tuning is set without timing anything;
    otherwise the sweep runs and its choice is stored under the key.  Returns
    (best, log, hit); log is empty on a hit."""
    import json
    import os
    path = default_cache_path() if path is None else path
    cache = _load(path)
    if key in cache:
        best = dict(h.get_tuning(), **{k: int(v) for k, v in cache[key].items() if k in h.TUNING_FIELDS})
        h.set_tuning(best)
        return h.get_tuning(), [], True
    best, log = tune(run, trials=trials, candidates=candidates, stream=stream)
    cache = _load(path)  # another process may have written meanwhile
    cache[key] = best
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return best, log, False
