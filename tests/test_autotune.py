"""Host logic of the launch-shape autotuner (no GPU: a fake timer)."""
from __future__ import annotations

import json

import numpy as np

from paper_2505_17368_gb300 import autotune


class _FakeIndex:
    n, d, storage = 1000, 32, 1


def test_candidates_follow_the_beam():
    c = autotune.candidates(10, 64)
    assert {"warps_per_block": 4, "team_size": 1, "hash_bits": 10} in c
    # team sizes 1, 2 and 4 warps per query, each dividing the block's warps
    assert {s["team_size"] for s in c} == {1, 2, 4}
    assert all(s["warps_per_block"] % s["team_size"] == 0 for s in c)
    assert all(8 <= s["hash_bits"] <= 15 for s in c)
    big = autotune.candidates(10, 512, ef_upper=64)
    assert max(s["hash_bits"] for s in big) > max(s["hash_bits"] for s in c)
    # the visited-table sort (exact_method 0) needs 2^(hash_bits - 1) slots
    # per exact-layer point; tiles and scans use none of them
    sort = autotune.candidates(10, 64, exact_upper=1000, exact_method=0)
    assert sort and all((1 << (s["hash_bits"] - 1)) >= 1000 for s in sort)
    tiles = autotune.candidates(10, 64, exact_upper=4000, exact_method=1)
    assert [dict(t) for t in tiles if t.pop("tile_n") == 256] == c  # each shape with 256- and 128-column tiles
    assert {t["tile_n"] for t in autotune.candidates(10, 64, exact_upper=4000, exact_method=1)} == {128, 256}
    assert autotune.candidates(10, 64, exact_upper=100000, exact_method=0) == []


def test_tune_picks_fastest_and_caches(tmp_path):
    Q = np.zeros((3000, 32), np.float32)
    calls = []

    def timer(shape):
        calls.append(shape)
        return (1.0 + 0.1 * shape["hash_bits"] - (0.5 if shape["warps_per_block"] == 2 else 0.0)
                - (0.2 if shape["team_size"] == 2 else 0.0))

    path = str(tmp_path / "cache.json")
    best = autotune.tune(_FakeIndex(), Q, k=10, ef=64, cache_path=path, timer=timer)
    assert best["warps_per_block"] == 2 and best["team_size"] == 2
    assert best["hash_bits"] == min(s["hash_bits"] for s in autotune.candidates(10, 64))
    n_first = len(calls)
    again = autotune.tune(_FakeIndex(), Q, k=10, ef=64, cache_path=path, timer=timer)
    assert again == best and len(calls) == n_first  # served from the cache
    data = json.load(open(path))
    (entry,) = data.values()
    assert entry["shape"] == best and len(entry["tried"]) == n_first
    # another batch bucket is tuned separately
    autotune.tune(_FakeIndex(), np.zeros((9000, 32), np.float32), k=10, ef=64, cache_path=path, timer=timer)
    assert len(json.load(open(path))) == 2
