"""Autotuner of the library's launch variants, launch shapes and cell size, with a JSON cache.

Three stages, each timed with CUDA events on the caller's own workload:
  1. ``rt_autotune`` (in the library) times every launch-variant combination of the float
     pair kernels (pair-flux variant, gather variant, gradient variant; all give the same
     result bits) and adopts the fastest;
  2. for the chosen variants, the threads per block of the gradient and the gather and the
     warps per block of the pair pass, one at a time (each also bitwise neutral), by timing
     sub-cycles through the library;
  3. the cell size of the neighbour search (its cell edge relative to the mean-density
     support radius), by timing ``rt_neighbours``; the pair lists do not depend on it.
The outcome is keyed by the workload's shape -- particles N, groups G, pairs P, Riemann
solver and precision -- and stored in a JSON file, so that later runs of the same shape
apply the cached choice without timing again.
"""
from __future__ import annotations

import json
import os

from . import rt_autotune, rt_diagnostics

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")


def shape_key(n: int, G: int, pairs: int, riemann: str, precision: str) -> str:
    return f"N={n};G={G};P={pairs};riemann={riemann};precision={precision}"


def load_cache(path: str) -> dict:
    if not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup_or_tune(key: str, tune, apply, cache_path: str = DEFAULT_CACHE, retune: bool = False) -> dict:
    """Apply the cached tuning for `key`, or call `tune()` -> (tuning, ms list), cache it and
    apply it.  Returns the cache entry ({"tuning": ..., "ms": ..., "source": ...})."""
    cache = load_cache(cache_path)
    entry = cache.get(key)
    if entry is not None and not retune:
        apply(entry["tuning"])
        return dict(entry, source="cache")
    tuning, ms = tune()
    entry = {"tuning": tuning, "ms": ms}
    cache[key] = entry
    store_cache(cache_path, cache)
    apply(tuning)
    return dict(entry, source="measured")


GRADIENT_BLOCKS = (32, 64, 128, 256)
GATHER_BLOCKS = (128, 256, 512)
PAIR_WARPS = (1, 2, 4)
CELL_EIGHTHS = (2, 3, 4, 6, 8)


def _time_ms(fn, repeats):
    """Shortest of `repeats` timings of fn() (CUDA events on the current stream), after one
    warm-up call."""
    import torch
    stream = torch.cuda.current_stream()
    best = None
    for r in range(repeats + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1)
        if r and (best is None or t < best):
            best = t
    return best


def tune_shapes(transport, U, dt, n_sub, L=None, alpha=None, repeats=2, tuning=None,
                subcycles_per_build=None) -> tuple:
    """Stages 2 and 3 from the variants in `tuning` (default: the context's): returns the
    tuning with the fastest shapes and cell size, and the times of every candidate.  The
    cell size sets the particle order, so it is scored by one rebuild plus the
    `subcycles_per_build` steps (default n_sub) that one build serves."""
    t = dict(tuning or transport.tuning())
    report = {}

    def steps():
        V = U.clone()
        for _ in range(n_sub):
            transport.step(V, dt, L, alpha)

    knobs = [("gradient_block", GRADIENT_BLOCKS)]
    if t["gather_variant"] == 1:
        knobs.append(("gather_block", GATHER_BLOCKS))
    if t["flux_variant"] == 2:
        knobs.append(("pair_warps", PAIR_WARPS))
    for knob, values in knobs:
        times = {}
        for v in values:
            transport.set_tuning(**dict(t, **{knob: v}))
            times[v] = _time_ms(steps, repeats)
        t[knob] = min(times, key=times.get)
        report[knob + "_ms"] = {str(k): v for k, v in times.items()}
    per_build = n_sub if subcycles_per_build is None else subcycles_per_build
    rebuild, stepping, score = {}, {}, {}
    P0 = transport.diagnostics()["n_pairs"]
    for ce in CELL_EIGHTHS:
        transport.set_tuning(**dict(t, cell_eighths=ce))
        rebuild[ce] = _time_ms(transport.rebuild, repeats)
        if transport.diagnostics()["n_pairs"] != P0:
            raise RuntimeError("the cell size changed the pair count")
        stepping[ce] = _time_ms(steps, repeats)
        score[ce] = rebuild[ce] + stepping[ce] * per_build / n_sub
    t["cell_eighths"] = min(score, key=score.get)
    report["cell_eighths_rebuild_ms"] = {str(k): v for k, v in rebuild.items()}
    report["cell_eighths_steps_ms"] = {str(k): v for k, v in stepping.items()}
    report["cell_eighths_score_ms"] = {str(k): v for k, v in score.items()}
    transport.set_tuning(**t)
    transport.rebuild()
    return t, report


def autotune(transport, U, dt, n_sub, L=None, alpha=None, repeats=3, cache_path: str = DEFAULT_CACHE,
             retune: bool = False, shapes: bool = True, subcycles_per_build=None) -> dict:
    """Tune a ``Transport`` on the device state U (torch tensor [G, 4, N]); n_sub steps
    are timed per candidate, and `subcycles_per_build` (default n_sub) weighs the steps
    against a rebuild when the cell size is chosen."""
    d = rt_diagnostics(transport.ctx)
    key = shape_key(transport.n, transport.G, d["n_pairs"], transport.riemann, transport.precision)

    def tune():
        transport._sync_stream()
        best, ms = rt_autotune(transport.ctx, U, dt, n_sub, L, alpha, repeats)
        report = {"variants_ms": ms}
        if shapes and transport.precision == "fp32":
            best, more = tune_shapes(transport, U, dt, n_sub, L, alpha, max(1, repeats - 1), best,
                                     subcycles_per_build)
            report.update(more)
        return best, report

    def apply(t):
        cur = transport.tuning()
        transport.set_tuning(**{k: t.get(k, cur[k]) for k in cur})
        if transport.tuning()["cell_eighths"] != cur["cell_eighths"]:
            transport.rebuild()

    out = lookup_or_tune(key, tune, apply, cache_path, retune)
    out["key"] = key
    return out
