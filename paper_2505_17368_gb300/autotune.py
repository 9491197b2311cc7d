"""Launch-shape autotuner for henn_search.

For an index, a batch size and a beam configuration, times henn_search over
a small grid of launch shapes -- warps per block, warps per query (the team
size: a team shares each expansion's distance work, which shortens a query
but leaves fewer queries in flight), the size of the per-query visited
table and, for an exact layer from tensor-core tiles, the tile's width
(128 x 128 or 128 x 256) -- and keeps the fastest.  Results are cached in a JSON file keyed by
(n, d, storage, batch bucket, k, ef, ef_upper, ef_l1, descend_all, exact
layer, rerank), so a process pays the sweep once per shape.  No knob
changes results: the visited table may forget entries without changing the
answer, a row's distance does not depend on which warp of a team computes
it nor a tile value on the tile's width, and queries are independent of the
grid.

    shape = autotune.tune(index, Q_device, k=10, ef=64, ef_upper=64)
    ids, d, _ = index.search(Q_device, k=10, ef=64, ef_upper=64, **shape)
"""
from __future__ import annotations

import json
import math
import os
import threading

_LOCK = threading.Lock()
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "henn_gb300_autotune.json")


def _beam_cap(k, ef, ef_upper, ef_l1):
    need = max(k, ef, ef_upper, ef_l1)
    cap = 32
    while cap < need:
        cap <<= 1
    return cap


def _default_hash_bits(cap):
    hb = 10
    while hb < 12 and (1 << hb) < cap * 8:
        hb += 1
    return hb


def candidates(k, ef, ef_upper=1, ef_l1=0, exact_upper=0, exact_method=0):
    """Shapes to try; exact_upper > 0 with exact_method 0 (SORT) needs
    2^(hash_bits - 1) >= exact_upper (the exact layer's keys use the visited
    table's space)."""
    hb = _default_hash_bits(_beam_cap(k, ef, ef_upper, ef_l1))
    need = exact_upper if exact_method == 0 else 0
    # the tensor-core tile shape of the batched exact layer (exact_method 1)
    tiles = (256, 128) if exact_method == 1 and exact_upper > 0 else (0,)
    out = []
    for w, t in ((4, 1), (2, 1), (4, 2), (2, 2), (4, 4)):
        for h in (hb - 2, hb - 1, hb, hb + 1):
            if 8 <= h <= 15 and (1 << (h - 1)) >= need:
                for n in tiles:
                    shape = {"warps_per_block": w, "team_size": t, "hash_bits": h}
                    if n:
                        shape["tile_n"] = n
                    out.append(shape)
    return out


def _key(index, nq, k, ef, ef_upper, ef_l1, descend_all, exact_upper=0, exact_method=0, rerank_mult=4):
    bucket = 1 << max(0, int(math.ceil(math.log2(max(nq, 1)))))
    return (f"n={index.n},d={index.d},s={index.storage},b={bucket},k={k},ef={ef},eu={ef_upper},l1={ef_l1},"
            f"da={descend_all},xu={exact_upper},xm={exact_method},rm={rerank_mult},v=team,tile")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _cuda_timer(index, Q, k, ef, ef_upper, ef_l1, descend_all, repeats, exact_upper=0, exact_method=0,
                rerank_mult=4):
    import torch

    def run(shape):
        shape = dict(shape, exact_upper=exact_upper, exact_method=exact_method, rerank_mult=rerank_mult)
        index.search(Q, k=k, ef=ef, ef_upper=ef_upper, ef_l1=ef_l1, descend_all=descend_all, **shape)
        torch.cuda.synchronize()
        ts = []
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            index.search(Q, k=k, ef=ef, ef_upper=ef_upper, ef_l1=ef_l1, descend_all=descend_all, **shape)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts)

    return run


def tune(index, Q, k=10, ef=64, ef_upper=1, ef_l1=0, descend_all=0, repeats=3, cache_path=DEFAULT_CACHE,
         use_cache=True, timer=None, exact_upper=0, exact_method=0, rerank_mult=4):
    """Fastest launch shape for this (index, batch, beam); Q is a CUDA
    tensor.  `timer(shape) -> ms` replaces the CUDA-event timing (tests)."""
    key = _key(index, Q.shape[0], k, ef, ef_upper, ef_l1, descend_all, exact_upper, exact_method, rerank_mult)
    with _LOCK:
        cache = _load(cache_path) if use_cache else {}
        if key in cache:
            return dict(cache[key]["shape"])
    run = timer or _cuda_timer(index, Q, k, ef, ef_upper, ef_l1, descend_all, repeats, exact_upper, exact_method,
                               rerank_mult)
    best, best_t, table = None, float("inf"), []
    for shape in candidates(k, ef, ef_upper, ef_l1, exact_upper, exact_method):
        t = run(shape)
        table.append((shape, t))
        if t < best_t:
            best, best_t = shape, t
    if use_cache:
        with _LOCK:
            cache = _load(cache_path)
            cache[key] = {"shape": best, "ms": best_t, "tried": [{"shape": s, "ms": t} for s, t in table]}
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            tmp = cache_path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, cache_path)
    return dict(best)
