"""Warp teams (team_size 2 and 4 warps per query): the team's warps share
the distance work of each beam expansion, and each row's distance is
computed by the same lane arithmetic whichever warp takes it, so results
(ids, distances and the per-query counters) are identical to one warp per
query, across storage forms, beam shapes, per-query k / ef and row widths."""
from __future__ import annotations

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_17368_gb300 as H  # noqa: E402

DEV = torch.device("cuda:0")


def _same_across_teams(idx, Q, **kw):
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(DEV)
    ref = [t.cpu().numpy() for t in idx.search(Qd, stats=True, team_size=1, **kw)]
    for team, warps in ((2, 4), (4, 4), (2, 2)):
        got = [t.cpu().numpy() for t in idx.search(Qd, stats=True, team_size=team, warps_per_block=warps, **kw)]
        for r, g in zip(ref, got):
            assert np.array_equal(r, g), (team, warps, kw)
    return ref


@pytest.fixture(scope="module")
def uniform():
    X, Q, _ = synth.workload("uniform-10k-d32")
    return H.Index(torch.from_numpy(X).to(DEV), seed=0), Q


@pytest.mark.parametrize("kw", [dict(k=10, ef=64), dict(k=10, ef=256), dict(k=10, ef=32, ef_upper=16, descend_all=1),
                                dict(k=10, ef=48, ef_upper=16, descend_all=1, exact_upper=700, exact_method=1)])
def test_team_sizes_give_identical_results(uniform, kw):
    idx, Q = uniform
    kw = dict(kw)
    if kw.get("exact_upper"):
        kw["exact_upper"] = idx.info()["sizes"][1]
    _same_across_teams(idx, Q, **kw)


def test_team_sizes_per_query_k_ef(uniform):
    idx, Q = uniform
    rng = np.random.default_rng(4)
    k = torch.from_numpy(rng.choice([1, 10, 37], size=len(Q)).astype(np.int32)).to(DEV)
    ef = torch.from_numpy(synth.log_uniform_int(len(Q), 16, 256, seed=5)).to(DEV)
    _same_across_teams(idx, Q, k=k, ef=ef, out_stride=40)


@pytest.mark.parametrize("storage,d", [(H.BF16, 128), (H.FP8E4M3, 128), (H.BF16, 960)])
def test_team_sizes_precision_forms_and_wide_rows(storage, d):
    X, r = synth.gaussian_mixture(8000, d, 40, seed=3, rescale_to_255=d == 128)
    Q, _ = synth.gaussian_mixture(500, d, 40, seed=4, rescale_from=r if d == 128 else None, rescale_to_255=d == 128)
    idx = H.Index(torch.from_numpy(X).to(DEV), storage=storage, seed=1)
    _same_across_teams(idx, Q, k=10, ef=64, ef_upper=8)


def test_team_size_must_divide_the_block(uniform):
    idx, Q = uniform
    for team, warps in ((3, 4), (4, 2)):
        with pytest.raises(H.HennError) as e:
            idx.search(Q[:10], k=10, ef=32, team_size=team, warps_per_block=warps)
        assert e.value.status == 1
