"""Host logic of bench.py (no GPU): the beam entries, the FP64 ground truth
and recall scoring, and the lookup of the search kernel's DRAM bytes in the
committed ncu summary."""
from __future__ import annotations

import hashlib
import os

import numpy as np
from scipy.spatial.distance import cdist

import bench
import synth


def test_default_and_walk_beams():
    ef, efu, da, l1, xu, xm, rm = bench.DEFAULT_BEAM
    assert ef >= bench.K and xm in (0, 1, 2) and rm >= 1
    assert not (xm != 0 and da and efu > 32)
    b = bench._beam(bench.DEFAULT_BEAM, [1000, 100, 37, 5])
    assert b[4] == 37 and all(isinstance(v, int) for v in b)
    assert bench._beam(bench.DEFAULT_BEAM, [1000, 100])[4] == 0  # no layer 2: no exact layer
    for entry in bench.WALK_SWEEP:
        assert entry[3] == 0  # the walk-only figure uses no exact layer


def test_fp64_ground_truth_matches_brute_force():
    """fp64_bruteforce (chunked, FP64 dot-product candidates re-ordered by
    direct differences) gives scipy's exact k nearest, ties by id; the
    re-ranking of a candidate pool that holds them gives the same."""
    X = synth.uniform_cube(5000, 12, seed=3)
    Q = synth.uniform_cube(60, 12, seed=4)
    X[17] = X[5]  # an exact tie: the smaller id first
    Q[0] = X[5]
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    want = np.array([np.lexsort((np.arange(len(X)), D[q]))[:10] for q in range(len(Q))])
    got_i, got_d = bench.fp64_bruteforce(X, Q, 10, pool=32, chunk=1300)
    assert np.array_equal(got_i, want)
    assert np.allclose(got_d, np.take_along_axis(D, want, 1), rtol=1e-12)
    pool = np.array([np.argsort(D[q], kind="stable")[:40] for q in range(len(Q))])[:, ::-1].copy()
    assert np.array_equal(bench.rerank_fp64(X, Q, pool, 10)[0], want)


def test_recall_fp64_counts_ties():
    X = np.array([[0.0], [1.0], [-1.0], [2.0], [3.0]], np.float32)
    Q = np.array([[0.0]], np.float32)
    gt_i, gt_d = bench.fp64_bruteforce(X, Q, 2, pool=5)
    assert gt_i.tolist() == [[0, 1]]
    assert bench.recall_fp64(X, Q, np.array([[0, 2]]), gt_i, gt_d) == 1.0  # -1 ties with the 2nd
    assert bench.recall_fp64(X, Q, np.array([[0, 3]]), gt_i, gt_d) == 0.5
    assert bench.recall_fp64(X, Q, np.array([[4, -1]]), gt_i, gt_d) == 0.0


def test_sweep_entries_are_well_formed():
    for entry in bench.UPPER_SWEEP:
        assert len(entry) in (5, 6), entry
        efu, da, l1, xu, xm = entry[:5]
        assert efu >= 0 and da in (0, 1) and l1 >= 0 and xm in (0, 1, 2)
        assert isinstance(xu, int) or (isinstance(xu, str) and xu[0] == "L" and xu[1:].isdigit())
        if xm != 0 and da:
            assert efu <= 32  # the tile and scan methods keep at most 32 seeds
        if len(entry) == 6:
            assert entry[5] >= 1
    assert bench.EF_SWEEP == sorted(bench.EF_SWEEP)


def _tree(tmp_path, src, lines):
    csrc = tmp_path / "paper_2505_17368_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "search.cu").write_bytes(src)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "search_bf16_mixture-1m-d128.md").write_text("# summary\n\n" + "".join(f"- {l}\n" for l in lines))


def test_profile_traffic_lookup(tmp_path, monkeypatch):
    src = b"// kernel source\n"
    sha = hashlib.sha256(src).hexdigest()[:16]
    _tree(tmp_path, src, [
        f"search.cu sha256[:16]: {sha}",
        "dram bytes per launch [ef=48 ef_upper=8 descend_all=1 ef_l1=0 exact_upper=3677 exact_method=1]: 111",
        "dram bytes per launch [ef=48 ef_upper=8 descend_all=1 ef_l1=0 exact_upper=3677 exact_method=1 "
        "rerank_mult=2]: 222",
    ])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    beam = (48, 8, 1, 0, 3677, 1)
    assert bench._profile_traffic(beam) == 111.0
    assert bench._profile_traffic(beam, 2) == 222.0
    assert bench._profile_traffic(beam, 3) is None
    assert bench._profile_traffic((44, 16, 1, 0, 3677, 1)) is None
    # a summary taken on another kernel source is not used
    (tmp_path / "paper_2505_17368_gb300" / "csrc" / "search.cu").write_bytes(src + b"// changed\n")
    assert bench._profile_traffic(beam) is None


def test_profile_traffic_without_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert not os.path.exists(tmp_path / "profiles")
    assert bench._profile_traffic((48, 8, 1, 0, 3677, 1)) is None


def test_serving_leg_reports_a_failure_instead_of_raising():
    """The serving measurement runs after the timed regions; a failure there
    (here a server that cannot be created) is reported in the line and the
    headline stands."""
    class _FakeH:
        class Server:
            def __init__(self, *a, **kw):
                raise RuntimeError("no serving kernel on this host")

    out = bench._serving_leg(_FakeH, index=None, Q=np.zeros((4, 128), np.float32), sizes=[1000, 100, 37, 5])
    assert out == {"error": "no serving kernel on this host"}
