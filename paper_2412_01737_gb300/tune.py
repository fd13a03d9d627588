"""Autotuner for the sampler's launch shape.

The tunable is the batch size k (`delay`): larger batches fold more links
into one tensor-core flush (fewer passes over W) but make the flush a
higher-rank product (k r), the small-matrix work of every link step grow
with (k r)^2, and the X application grow with N (k r)^2; the panels cost
2 k r N and the small matrices 2 (k r)^2 of memory per pair and chain.  For a given problem and chain count the tuner times one
sweep per candidate through the C ABI and keeps the fastest; results are
cached in a JSON file keyed by (lattice, group, n_v, K, chains, precision).
"""
from __future__ import annotations

import json
import os
import time

DEFAULT_CANDIDATES = (4, 8, 16)


def cache_path() -> str:
    return os.environ.get("GGF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ggf_tune.json"))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key_of(p, chains, precision) -> str:
    return f"L{p.L}_g{p.group}_nv{p.n_v}_K{p.K}_c{chains}_p{precision}"


def tune_delay(p, links, precision, device=0, candidates=DEFAULT_CANDIDATES, use_cache=True, seed=1):
    """Best delay for `p` with the starting links `links` (host array).
    Returns (delay, {candidate: ms per sweep})."""
    import torch
    from .ggf import GGF, GGFError
    path = cache_path()
    key = key_of(p, len(links), precision)
    cache = _load(path) if use_cache else {}
    if key in cache:
        return int(cache[key]["delay"]), {int(k): v for k, v in cache[key]["ms"].items()}
    timings = {}
    for d in candidates:
        ctx = GGF(device)
        try:
            ctx.init_problem(p)
            ctx.chains_init(links, precision=precision, refresh_every=1 << 30, seed=seed, delay=d)
            ctx.sample(1)                              # graph capture and warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.sample(1)
            torch.cuda.synchronize()
            timings[d] = 1e3 * (time.perf_counter() - t0)
        except GGFError:
            timings[d] = float("inf")                  # e.g. panels do not fit
        finally:
            ctx.close()
    best = min(timings, key=timings.get)
    if use_cache:
        cache[key] = {"delay": best, "ms": {str(k): v for k, v in timings.items()}}
        _store(path, cache)
    return best, timings
