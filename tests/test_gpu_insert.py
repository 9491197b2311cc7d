"""Dynamic Insert (App. C) on the GPU against the oracle's Insert."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_2505_17368_gb300 as H  # noqa: E402
import synth  # noqa: E402

from test_gpu_parity import DEV, _gpu_index, _graph_parity, _layers_equal  # noqa: E402
from tests import parity as P  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_insert_parity(storage):
    """Points appended by henn_insert (in two calls, so the arrays grow)
    land in the same layers as the oracle's Insert, with the same forward
    lists and adjacency (up to near-ties), and a search for an inserted
    point returns it first."""
    X = synth.uniform_cube(5200, 16, seed=41)
    oidx = O.build_index(X[:4000], seed=6)
    st = H.F32 if storage == "f32" else H.BF16
    gidx = _gpu_index(X[:4000], seed=6, storage=st)
    O.insert(oidx, X, np.arange(4000, 5200))
    assert gidx.insert(X[4000:4600]) == 4000
    assert gidx.insert(torch.from_numpy(X[4600:]).to(DEV)) == 4600
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X)
    q = np.arange(4000, 5200, 37)
    ids, dd, _ = gidx.search(torch.from_numpy(X[q]).to(DEV), k=1, ef=64)
    assert np.array_equal(ids.cpu().numpy()[:, 0], q)
    assert np.all(dd.cpu().numpy()[:, 0] == 0)


def test_insert_rejects_knn_graphs():
    X = synth.uniform_cube(1000, 8, seed=2)
    gidx = _gpu_index(X, graph=H.GRAPH_KNN, seed=1)
    with pytest.raises(H.HennError) as e:
        gidx.insert(X[:10])
    assert e.value.status == 6


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_delete_parity(storage):
    """Delete as tombstones: deleted points never come back, and recall
    against the live points' exact neighbours tracks the oracle's."""
    X = synth.uniform_cube(6000, 16, seed=43)
    Q = synth.uniform_cube(1500, 16, seed=44)
    st = H.F32 if storage == "f32" else H.BF16
    oidx = O.build_index(X, seed=9)
    gidx = _gpu_index(X, seed=9, storage=st)
    dead = np.zeros(len(X), bool)
    dead[::4] = True
    gi_all, _ = O.bruteforce(X, Q, 1)
    dead[gi_all[:400, 0]] = True  # some queries lose their nearest point
    gidx.delete(np.nonzero(dead)[0][: len(np.nonzero(dead)[0]) // 2])
    gidx.delete(np.nonzero(dead)[0][len(np.nonzero(dead)[0]) // 2:])
    ids, dd, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=64)
    ids = ids.cpu().numpy()
    oi, od, _ = O.search(oidx, X, Q, k=10, ef=64, deleted=dead)
    assert np.all(ids >= 0) and not dead[ids].any()
    live = np.nonzero(~dead)[0]
    li, ld = O.bruteforce(X[live], Q, 10)
    gt = live[li]
    rec = lambda found: np.mean([len(set(found[q]) & set(gt[q])) / 10 for q in range(len(Q))])  # noqa: E731
    print(f"delete {storage}: gpu {rec(ids):.4f} oracle {rec(oi):.4f}")
    assert abs(rec(ids) - rec(oi)) <= P.RECALL_TOL + 1e-12, (rec(ids), rec(oi))
    assert np.all(np.diff(dd.cpu().numpy(), axis=1) >= 0)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_delete_resampling_parity(storage):
    """Delete of App. C with resampling: the GPU and the oracle apply the
    same deletions (two calls, the first too small to trigger anything);
    when layer 1's live part falls below half of a fresh sample of the live
    base, both resample it from the live points and rebuild above it.  The
    layers are bit-exact, the graphs match up to near ties, deleted points
    never come back, and recall on the live points tracks the oracle's."""
    X = synth.uniform_cube(8000, 16, seed=71)
    Q = synth.uniform_cube(1500, 16, seed=72)
    st = H.F32 if storage == "f32" else H.BF16
    oidx = O.build_index(X, seed=12)
    gidx = _gpu_index(X, seed=12, storage=st)
    l1 = oidx["ids"][1].copy()
    dead = np.zeros(len(X), bool)
    first = np.concatenate([l1[:4], np.arange(0, len(X), 97)])
    dead[first] = True
    gidx.delete(first)
    assert O.delete(oidx, X, dead) is None
    _layers_equal(gidx, oidx)
    second = np.concatenate([l1[: (2 * len(l1)) // 3], np.arange(5, len(X), 11)])
    dead[second] = True
    gidx.delete(second)
    assert O.delete(oidx, X, dead) == 1
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X)
    for i in range(1, gidx.info()["L"] + 1):
        assert not dead[gidx.layer(i)["ids"]].any()
    ids, dd, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=64)
    ids = ids.cpu().numpy()
    assert np.all(ids >= 0) and not dead[ids].any()
    oi, _, _ = O.search(oidx, X, Q, k=10, ef=64, deleted=dead)
    live = np.nonzero(~dead)[0]
    li, _ = O.bruteforce(X[live], Q, 10)
    gt = live[li]
    rec = lambda found: np.mean([len(set(found[q]) & set(gt[q])) / 10 for q in range(len(Q))])  # noqa: E731
    print(f"delete+resample {storage}: gpu {rec(ids):.4f} oracle {rec(oi):.4f}")
    assert abs(rec(ids) - rec(oi)) <= P.RECALL_TOL + 1e-12, (rec(ids), rec(oi))
