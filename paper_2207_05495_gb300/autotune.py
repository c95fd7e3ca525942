"""Autotuner for the search's tunable parameters (sw_options).

It times the batched search on a sample of automata for every candidate
setting of the meet kernel's forward rows per tile and backward chunk size
(lane words) and of the direction rule (SetCost, the threshold theta of the
step-cost comparison and its meet term, pair count or ExpMark, Section
2.1.2); the inclusion reductions (Alg. 1) can be added to a grid.  A setting
whose warm-up run on an eighth of the sample already takes longer than the
best whole-sample time so far is dropped without timing, and tuning stops
at a time limit with the best setting found.  It requires every candidate
to return identical r, and identical words among
the candidates without reductions (with a reduced side the word depends on
the depth at which the two searches met, so there each word must only
reset the automaton and have length r), and keeps the fastest.  Results are cached in tuned.json next to this file,
keyed by (words per set W, letters k, GPU name); `apply` loads the entry for
a workload into the calling thread's options.

    python -m paper_2207_05495_gb300.autotune   # tunes the 4096-automaton workload's shape
"""

from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

from . import gen, sw

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")

# The reductions are left out of the default grid: on random automata of
# 64..192 states they cost several times what they save (marking is
# quadratic in the candidates), so they are only worth a grid of their own
# for single hard instances.
GRID = {
    "meet_f_rows": [4096, 16384],
    "meet_lane_words": [0, 4],
    "set_cost": [128.0, 512.0, 8192.0, 131072.0],
    "dir_theta": [0.5, 1.0, 2.0],
    "dir_rule": [0, 1],
}


def key(W: int, k: int, gpu: str) -> str:
    return f"W{W}-k{k}-{gpu}"


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(0)


def _resets(delta: np.ndarray, word) -> bool:
    states = np.arange(delta.shape[1])
    for a in word:
        states = delta[a][states]
    return len(np.unique(states)) == 1


def tune(automata, ws, grid=None, repeats: int = 2, verbose: bool = False, time_limit: float = 600.0) -> dict:
    """Times sw_batch over `automata` for every combination in `grid`
    (dict of option name -> values) until `time_limit` seconds have passed;
    returns {"best": {...}, "trials": [...], "pruned": n, "complete": bool}."""
    import torch
    grid = grid or GRID
    hs = [sw.load(d) for d in automata]
    base = sw.sw_get_options()
    names = list(grid)
    ref_r = None
    ref_words = None  # of the candidates without reductions
    trials = []
    pruned = 0
    complete = True
    t_start = time.perf_counter()
    best_so_far = None
    try:
        for combo in itertools.product(*(grid[n] for n in names)):
            if time.perf_counter() - t_start > time_limit:
                complete = False
                break
            o = sw.sw_get_options()
            for n, v in zip(names, combo):
                setattr(o, n, v)
            sw.sw_set_options(o)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sw.sw_batch(hs[: max(1, len(hs) // 8)], ws=ws)  # warm
            torch.cuda.synchronize()
            if best_so_far is not None and time.perf_counter() - t0 > best_so_far:
                pruned += 1
                continue
            best_t = None
            for _ in range(repeats):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r, w = sw.sw_batch(hs, ws=ws)
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
                best_t = t if best_t is None else min(best_t, t)
            red = int(getattr(o, "reduce", 0))
            if ref_r is None:
                ref_r = r.copy()
            if not (r == ref_r).all():
                raise RuntimeError(f"setting {dict(zip(names, combo))} changed r")
            if red == 0:
                if ref_words is None:
                    ref_words = w
                if w != ref_words:
                    raise RuntimeError(f"setting {dict(zip(names, combo))} changed the words")
            elif not all(len(wi) == ri and _resets(d, wi) for d, wi, ri in zip(automata, w, r)):
                raise RuntimeError(f"setting {dict(zip(names, combo))} returned a word that does not reset")
            trial = dict(zip(names, combo))
            trial["seconds"] = best_t
            trials.append(trial)
            best_so_far = best_t if best_so_far is None else min(best_so_far, best_t)
            if verbose:
                print(trial, flush=True)
    finally:
        sw.sw_set_options(base)
    best = min(trials, key=lambda t: t["seconds"])
    return {"best": {n: best[n] for n in names}, "seconds": best["seconds"], "trials": trials, "pruned": pruned,
            "complete": complete}


def load_cache() -> dict:
    if os.path.exists(CACHE):
        with open(CACHE) as fh:
            return json.load(fh)
    return {}


def save(entry_key: str, result: dict) -> None:
    cache = load_cache()
    cache[entry_key] = {"options": result["best"], "seconds": result["seconds"],
                        "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    with open(CACHE, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)


def apply(W: int, k: int) -> dict | None:
    """Sets the calling thread's options from the cache entry for (W, k, this
    GPU); returns the options applied, or None when there is no entry."""
    entry = load_cache().get(key(W, k, _gpu_name()))
    if not entry:
        return None
    o = sw.sw_get_options()
    for n, v in entry["options"].items():
        setattr(o, n, type(getattr(o, n))(v))
    sw.sw_set_options(o)
    return entry["options"]


def main():
    import torch
    from . import build
    build.build()
    torch.cuda.set_device(0)
    sample = gen.batch_random(512, 64, 192, 2, 0)
    W = max((d.shape[1] + 63) // 64 for d in sample)
    ws = sw.workspace(96 << 30)
    res = tune(sample, ws, verbose=True, time_limit=300.0)
    save(key(W, 2, _gpu_name()), res)
    print(json.dumps({"key": key(W, 2, _gpu_name()), "best": res["best"], "seconds": res["seconds"],
                      "trials": len(res["trials"]), "pruned": res["pruned"], "complete": res["complete"]}))


if __name__ == "__main__":
    main()
