"""Autotuner of the batched form: block size b (and with it the engine's column
tile BN = 8 * ceil(b / 8) rounded to a power of two) per problem shape.

Shapes are bucketed by (N rounded to a power of two, d, r rounded to 64).  For
each bucket one representative problem is factorised through the batched
launch with every candidate b that divides into at least one round, and the b
with the most accepted pivots per millisecond of kernel-column engine time
wins (measured with the library's tracer on single-problem runs).  The
per-round latency of the small launches (proposal, gather, block H, reject) is
left out of the score because a batch pays it once for all problems.  Results are cached in a JSON
file (KEVD_AUTOTUNE_CACHE, default ~/.cache/kevd/autotune.json) keyed by the
bucket and the GPU name.
"""
import json
import math
import os

import torch

from .kevd import rpchol_factor, trace_enable, trace_reset, trace_read

CANDIDATES = (16, 32, 64, 128)


def _cache_path():
    return os.environ.get("KEVD_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "kevd",
                                                              "autotune.json"))


def shape_key(N, d, r):
    nb = 1 << int(round(math.log2(max(N, 1))))
    return "N%d_d%d_r%d" % (nb, d, int(round(r / 64.0)) * 64)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, cache):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _time_one(prob, b, reps=2):
    """Accepted pivots per millisecond of engine time for block size b."""
    args = (prob["X"], prob["eps"], prob["r"])
    rpchol_factor(*args, mode="arpc", b=b, seed=prob.get("seed", 0))      # warm-up
    was = trace_enable(True)
    trace_reset()
    rank = 0
    for _ in range(reps):
        rank = rpchol_factor(*args, mode="arpc", b=b, seed=prob.get("seed", 0))["rank"]
    ms = trace_read()["engine"][0] / reps
    trace_enable(was)
    trace_reset()
    return rank / max(ms, 1e-6)


def tune(problems, candidates=CANDIDATES, use_cache=True):
    """Block size per problem (list of ints); problems are dicts as for Batch."""
    gpu = torch.cuda.get_device_name(problems[0]["X"].device)
    path = _cache_path()
    cache = _load(path) if use_cache else {}
    choice = []
    for p in problems:
        N, d = p["X"].shape
        key = "%s|%s" % (gpu, shape_key(N, d, p["r"]))
        if key not in cache:
            best, best_rate = None, -1.0
            for b in candidates:
                if b > p["r"] or b > 128:
                    continue
                rate = _time_one(p, b)
                if rate > best_rate:
                    best, best_rate = b, rate
            cache[key] = {"b": best, "pivots_per_s": best_rate}
        choice.append(int(cache[key]["b"]))
    if use_cache:
        _save(path, cache)
    return choice
