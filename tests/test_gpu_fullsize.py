"""The benchmarked configuration at full size (1M x 128 mixture, the bench's
default beam) against the FP64 oracle searching the same GPU-built
hierarchy (imported layers, down pointers and graphs), on sampled queries
scored against FP64 brute force (Sec. 2.2 query, Alg. 4 descent with the
candidate sets of readings 11 and 16).

Tolerances (tests/parity.py): recall@10 within 0.5 points of the oracle's
at the same beam, both directions; returned distances within 1e-4 of FP64.
"""
from __future__ import annotations

import numpy as np
import pytest

import bench
import oracle as O
import synth
from tests import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_17368_gb300 as H  # noqa: E402

DEV = torch.device("cuda:0")
NQ = 2000


@pytest.fixture(scope="module")
def full():
    X, Q, _ = synth.workload("mixture-1m-d128")
    sel = np.sort(np.random.default_rng(21).choice(len(Q), NQ, replace=False))
    Qs = np.ascontiguousarray(Q[sel])
    Xd = torch.from_numpy(X).to(DEV)
    g_bf16 = H.Index(Xd, storage=H.BF16, seed=0)
    g_f32 = H.Index(Xd, storage=H.F32, seed=0)
    del Xd
    view = P.oracle_view(g_bf16)
    O.set_threads(len(__import__("os").sched_getaffinity(0)))
    gi, gd = O.bruteforce(X, Qs, 10)
    return dict(X=X, Q=Qs, bf16=g_bf16, f32=g_f32, view=view, gi=gi, gd=gd)


def _gpu(index, Qs, beam):
    ef, efu, da, l1, xu, xm, rm = beam
    ids, dd, _ = index.search(torch.from_numpy(Qs).to(DEV), k=10, ef=ef, ef_upper=efu, descend_all=da, ef_l1=l1,
                              exact_upper=xu, exact_method=xm, rerank_mult=rm)
    return ids.cpu().numpy(), dd.cpu().numpy()


def _oracle(full, beam):
    ef, efu, da, l1, xu, _, _ = beam
    return O.search(full["view"], full["X"], full["Q"], k=10, ef=ef, ef_upper=efu, descend_all=da, ef_l1=l1,
                    exact_upper=xu)


def _check(full, ids, dd, oi):
    X, Qs, gi, gd = full["X"], full["Q"], full["gi"], full["gd"]
    rg = O.recall_at_k(ids, gi, gd).mean()
    ro = O.recall_at_k(oi, gi, gd).mean()
    assert abs(rg - ro) <= P.RECALL_TOL + 1e-12, (rg, ro)
    assert P.returned_distance_error(X, Qs, ids, dd) <= P.DIST_RTOL
    return rg, ro


def test_hierarchy_is_the_same_for_both_storage_forms(full):
    """Storage changes the traversal copies only: the BF16 and FP32 builds
    have the same layers and graphs, so one oracle view serves both."""
    a, b = full["bf16"].info(), full["f32"].info()
    assert a["sizes"] == b["sizes"]
    for i in range(a["L"] + 1):
        la, lb = full["bf16"].layer(i), full["f32"].layer(i)
        assert np.array_equal(la["adj"], lb["adj"]) and np.array_equal(la["ids"], lb["ids"]), i


def test_benchmarked_beam_bf16_tracks_oracle(full):
    """The bench's chosen form: BF16 traversal, the exact candidate set of
    layer 2 from distance tiles seeding a layer-1 beam, the layer-0 beam
    and the FP32 rerank -- against the oracle's FP64 search at the same
    beam on the same graphs."""
    beam = bench._beam(bench.DEFAULT_BEAM, full["bf16"].info()["sizes"])
    assert beam[4] > 0 and beam[5] == H.EXACT_TILES
    ids, dd = _gpu(full["bf16"], full["Q"], beam)
    oi, _, _ = _oracle(full, beam)
    rg, ro = _check(full, ids, dd, oi)
    print(f"bf16 default beam {beam}: gpu {rg:.4f} oracle {ro:.4f}")


def test_benchmarked_beam_f32_matches_oracle(full):
    """The same beam in FP32: besides recall, the answers themselves agree
    query by query up to FP32-against-FP64 near ties."""
    beam = bench._beam(bench.DEFAULT_BEAM, full["f32"].info()["sizes"])
    ids, dd = _gpu(full["f32"], full["Q"], beam)
    oi, _, _ = _oracle(full, beam)
    _check(full, ids, dd, oi)
    assert np.mean(np.all(ids == oi, axis=1)) >= 0.99


@pytest.mark.parametrize("beam", [(64, 64, 0, 16, 0, 0, 4), (96, 1, 0, 0, 0, 0, 4)])
def test_walked_upper_layers_track_oracle(full, beam):
    """Upper layers walked by beams only (reading 11), and the plain greedy
    descent of Alg. 4 (ef_upper 1), BF16 with the FP32 rerank."""
    ids, dd = _gpu(full["bf16"], full["Q"], beam)
    oi, _, _ = _oracle(full, beam)
    rg, ro = _check(full, ids, dd, oi)
    print(f"bf16 beam {beam}: gpu {rg:.4f} oracle {ro:.4f}")
