"""Autotuner for the plans' tile and split choices.

For a plan and a representative call it tries every candidate setting of the
knobs exposed by ``ndft_set_tuning`` (split count along the sample axis, tile
rows of the tensor-core form, tensor-memory accumulation chain length), times
each with CUDA events on the current stream, keeps the fastest and records it
in a JSON cache keyed by GPU name and problem shape, so later plans of the
same shape reuse the choice without timing.

Only settings that keep the accuracy bar are offered: the default chain
length of each contraction variant (0: 256 MMA K steps per chain, 64 blocks of
16 samples in the conjugate-paired one or of 8 samples in the unpaired one;
4.0e-6 / 4.9e-6 of max|X| on the worst case measured, the N = 2^18 NDFT of
CN(0,1) vectors) or shorter ones.
The cache lives at ``$NDFT_AUTOTUNE_CACHE`` or ``~/.cache/ndft_gb300/autotune.json``.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

_lock = threading.Lock()

SPLIT, ROWS, CHUNK, DRAIN = 0, 1, 2, 3
PARTS = 5  # tensor-core calls of >= 512 columns: 1 one part (default), 0 two parts (not tuned: see tune_caf)

TERNARY_SPACE = {ROWS: [256, 128, 258], CHUNK: [0, 64, 32], SPLIT: [0, 8, 16, 19, 24, 32]}
DIRECT_SPACE = {SPLIT: [0, 2, 4, 6, 8, 12, 16]}
# batched tensor-core plans: one persistent contraction over all CPIs, no split;
# the knobs are the chain length and the fold-out path
BATCHED_SPACE = {CHUNK: [64, 32], DRAIN: [0, 1]}


def cache_path() -> str:
    p = os.environ.get("NDFT_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "ndft_gb300", "autotune.json")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(space: dict) -> list[dict]:
    keys = sorted(space)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(space[k] for k in keys))]


def select(times: list[tuple[dict, float]]) -> dict:
    """The fastest setting; ties go to the earlier (default-first) candidate."""
    best, best_t = None, float("inf")
    for setting, t in times:
        if t < best_t * (1 - 1e-3):
            best, best_t = setting, t
    return best


def tune(plan, run, key: str, space: dict, device_name: str, reps: int = 3, timer=None, path: str | None = None,
         force: bool = False, rounds: int = 2) -> dict:
    """Pick the fastest setting of `space` for `run()` on `plan`, cached under (device, key).

    `timer(run, reps)` returns seconds per call (default: CUDA events around the
    calls); every candidate is timed in each of `rounds` passes over the space
    and keeps its best time, so a transient slowdown during one pass does not
    decide the choice.  The chosen setting is applied to the plan and returned."""
    path = path or cache_path()
    ckey = f"{device_name}|{key}"
    with _lock:
        cache = _load(path)
    if not force and ckey in cache:
        setting = {int(k): v for k, v in cache[ckey]["setting"].items()}
        for k, v in setting.items():
            plan.set_tuning(k, v)
        return setting
    timer = timer or _cuda_timer
    cands = candidates(space)
    best_t = [float("inf")] * len(cands)
    for r in range(max(1, rounds)):
        for i, setting in enumerate(cands):
            for k, v in setting.items():
                plan.set_tuning(k, v)
            if r == 0:
                run()  # warm
            best_t[i] = min(best_t[i], timer(run, reps))
    results = list(zip(cands, best_t))
    best = select(results)
    for k, v in best.items():
        plan.set_tuning(k, v)
    with _lock:
        cache = _load(path)
        cache[ckey] = {"setting": {str(k): v for k, v in best.items()},
                       "seconds": min(t for _, t in results), "tried": len(results)}
        _store(path, cache)
    return best


def _cuda_timer(run, reps: int) -> float:
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        run()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / 1000.0 / reps


def tune_batched(bplan, surv, ref, out, **kw) -> dict:
    """Tune a batched tensor-core plan on its own CPI list (one call = all CPIs)."""
    import torch
    key = f"batched|{bplan.form}|{bplan.prec}|{bplan.signature()}"
    name = torch.cuda.get_device_name(surv.device)
    return tune(bplan, lambda: bplan(surv, ref, out), key, BATCHED_SPACE, name, **kw)


def tune_caf(plan, s_surv, s_ref, lag0: int, nlags: int, out=None, **kw) -> dict:
    """Tune a CAF plan on one representative call."""
    import torch
    space = TERNARY_SPACE if plan.form == "ternary" else DIRECT_SPACE
    key = f"caf|{plan.form}|{plan.prec}|N={plan.n}|bins={plan.nbins}|lags={nlags}"
    out = out if out is not None else torch.empty(
        (nlags,) + plan._row_shape(plan.nbins), dtype=plan._out_dtype, device=s_surv.device)
    name = torch.cuda.get_device_name(s_surv.device)
    # (column parts are not tuned: two parts win the short timings here but lose
    # about 3 % in long runs at the power limit)
    return tune(plan, lambda: plan.caf(s_surv, s_ref, lag0, nlags, out=out), key, space, name, **kw)
