"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes span many tiles and ragged tails; the 1M x 128 workload that bench.py
times is checked on sampled rows and queries the oracle computes one by
one.  Tolerances: tests/parity.py.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import synth
from tests import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_17368_gb300 as H  # noqa: E402

DEV = torch.device("cuda:0")


def _gpu_index(X, **kw):
    return H.Index(torch.from_numpy(np.ascontiguousarray(X)).to(DEV), **kw)


def _layers_equal(gidx, oidx):
    info = gidx.info()
    assert info["L"] == oidx["L"], (info["sizes"], oidx["sizes"])
    assert info["sizes"] == [len(a) for a in oidx["ids"]]
    assert info["attempts"] == [int(a) for a in oidx["attempts"]]
    for i in range(1, info["L"] + 1):
        lay = gidx.layer(i)
        assert np.array_equal(lay["ids"], oidx["ids"][i]), f"layer {i} ids"
        assert np.array_equal(lay["down"], oidx["down"][i]), f"layer {i} down"
    return info


def _graph_parity(gidx, oidx, X, metric=0):
    tot_e = tot_ex = 0
    for i in range(oidx["L"] + 1):
        lay = gidx.layer(i)
        ids = oidx["ids"][i]
        e, ex, un, pairs = P.compare_rows(lay["fwd"], oidx["fwd"][i], X, ids, metric)
        assert un == 0, f"layer {i}: {un} unexcused forward-list differences"
        # forward distances: FP32 exact vs FP64
        ok = oidx["fwd"][i] >= 0
        same = ok & (lay["fwd"] == oidx["fwd"][i])
        g = lay["fwd_d"][same].astype(np.float64)
        o = oidx["fwd_d"][i][same]
        if metric == 1:
            o = o  # 1 - cos in both
        assert np.all(np.abs(g - o) <= 1e-4 * np.maximum(np.abs(o), 1e-6)), f"layer {i} forward distances"
        e2, ex2, un2 = P.compare_adjacency(lay["adj"], oidx["adj"][i], lay["fwd"], oidx["fwd"][i], pairs, X, ids, metric)
        assert un2 == 0, f"layer {i}: {un2} unexcused adjacency differences"
        tot_e += e + e2
        tot_ex += ex + ex2
    assert tot_ex <= P.EXCUSED_BUDGET * tot_e, (tot_ex, tot_e)
    return tot_ex, tot_e


@pytest.fixture(scope="module")
def uniform10k():
    X, Q, _ = synth.workload("uniform-10k-d32")
    oidx = O.build_index(X, seed=0)
    gidx = _gpu_index(X, seed=0)
    return X, Q, oidx, gidx


def test_graph_parity_simt_tiles(uniform10k):
    """The CUDA-core FP32 tile engine (used for d > 128) on the same layers."""
    X, Q, oidx, _ = uniform10k
    gidx = _gpu_index(X, seed=0, tiles=H.TILES_SIMT)
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X)


# ----------------------------------------------------------- layers

def test_layers_bit_exact_uniform10k(uniform10k):
    X, Q, oidx, gidx = uniform10k
    info = _layers_equal(gidx, oidx)
    assert info["L"] >= 2


@pytest.mark.parametrize("case", ["retries", "m2", "angular", "tiny", "oddd"])
def test_layers_bit_exact_cases(case):
    if case == "retries":  # small c0: several Las-Vegas attempts per layer
        X = synth.uniform_cube(4000, 8, seed=5)
        kw = dict(eps_c0=0.06, num_ranges=60, max_attempts=2000, seed=1)
        okw = dict(c0=0.06, r=60, max_attempts=2000, seed=1)
    elif case == "m2":
        X = synth.uniform_cube(5000, 16, seed=6)
        kw, okw = dict(m=2, seed=3), dict(m=2, seed=3)
    elif case == "angular":
        X, _ = synth.gaussian_mixture(6000, 96, 50, seed=0, normalise=True)
        kw = dict(metric=H.ANGULAR, eps_c0=0.02, seed=2)
        okw = dict(metric=O.ANGULAR, c0=0.02, seed=2)
    elif case == "tiny":
        X = synth.uniform_cube(40, 3, seed=7)
        kw, okw = dict(seed=4, eps_c0=0.2), dict(seed=4, c0=0.2)
    else:  # d not a multiple of 32, ragged tiles
        X = synth.uniform_cube(3001, 45, seed=8)
        kw, okw = dict(seed=5, eps_c0=0.05), dict(seed=5, c0=0.05)
    oidx = O.build_layers(X, **okw)
    gidx = _gpu_index(X, **kw)
    _layers_equal(gidx, oidx)
    if case == "retries":
        info = gidx.info()
        assert max(info["attempts"]) >= 1
        # the attempts relaunch one executable graph, updated in place
        assert info["graph_updates"] >= sum(info["attempts"]) and info["graph_instantiations"] <= 2 * info["L"] + 2


def test_epsnet_not_found_is_reported():
    X = synth.uniform_cube(4000, 8, seed=5)
    with pytest.raises(H.HennError) as e:
        _gpu_index(X, eps_c0=0.002, num_ranges=200, max_attempts=2, seed=1)
    assert e.value.status == 4


# ------------------------------------------------------------ graphs

def test_graph_parity_uniform10k(uniform10k):
    X, Q, oidx, gidx = uniform10k
    _graph_parity(gidx, oidx, X)


@pytest.mark.parametrize("case", ["knn", "mixture", "angular", "oddd"])
def test_graph_parity_cases(case):
    if case == "knn":
        X = synth.uniform_cube(3000, 24, seed=9)
        kw, okw = dict(graph=H.GRAPH_KNN, seed=6), dict(graph=O.GRAPH_KNN, seed=6)
        metric = 0
    elif case == "mixture":
        X, _ = synth.gaussian_mixture(8000, 128, 100, seed=0, rescale_to_255=True)
        kw, okw, metric = dict(seed=7), dict(seed=7), 0
    elif case == "angular":
        X, _ = synth.gaussian_mixture(6000, 96, 50, seed=0, normalise=True)
        kw = dict(metric=H.ANGULAR, seed=8)
        okw = dict(metric=O.ANGULAR, seed=8)
        metric = 1
    else:
        X = synth.uniform_cube(3001, 45, seed=8)
        kw, okw, metric = dict(seed=5), dict(seed=5), 0
    oidx = O.build_index(X, **okw)
    gidx = _gpu_index(X, **kw)
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X, metric)


@pytest.mark.parametrize("case", ["uniform", "mixture", "knn", "ragged", "d136", "d200", "d960"])
def test_graph_parity_tcgen05_tiles(case):
    """The tensor-core tile engine (tcgen05, split BF16) feeds the same
    exact rerank: forward lists and adjacency match the oracle.  Rows wider
    than 128 values (d136: 3 slices of 64, d200: 4, d960: 15) stream the
    row block through the pipeline instead of keeping it resident."""
    if case == "d136":
        X = synth.uniform_cube(3001, 136, seed=12)
        kw, okw = dict(seed=4), dict(seed=4)
    elif case == "d200":
        X, _ = synth.gaussian_mixture(5000, 200, 60, seed=1, rescale_to_255=True)
        kw, okw = dict(seed=3), dict(seed=3)
    elif case == "d960":
        X, _ = synth.gaussian_mixture(4000, 960, 40, seed=2)
        kw, okw = dict(seed=2), dict(seed=2)
    elif case == "uniform":
        X = synth.uniform_cube(10000, 32, seed=0)
        kw, okw = dict(seed=0), dict(seed=0)
    elif case == "mixture":
        X, _ = synth.gaussian_mixture(12000, 128, 100, seed=0, rescale_to_255=True)
        kw, okw = dict(seed=7), dict(seed=7)
    elif case == "knn":
        X = synth.uniform_cube(3000, 24, seed=9)
        kw, okw = dict(graph=H.GRAPH_KNN, seed=6), dict(graph=O.GRAPH_KNN, seed=6)
    else:  # rows not a multiple of the 128 x 256 tile, d not a multiple of 64
        X = synth.uniform_cube(3001, 45, seed=8)
        kw, okw = dict(seed=5), dict(seed=5)
    oidx = O.build_index(X, **okw)
    gidx = _gpu_index(X, tiles=H.TILES_TCGEN05, **kw)
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X)


def _lattice(side, dim, pad_to=None):
    g = np.stack(np.meshgrid(*[np.arange(side)] * dim, indexing="ij"), -1).reshape(-1, dim).astype(np.float32)
    g = g[np.random.default_rng(3).permutation(len(g))]
    if pad_to:
        g = np.concatenate([g, np.zeros((len(g), pad_to - dim), np.float32)], axis=1)
    return np.ascontiguousarray(g)


@pytest.mark.parametrize("case", ["nsw_tc", "nsw_simt", "knn", "wide", "d96"])
def test_graph_parity_uncertified_rows(case):
    """Integer lattices put many points at exactly the M-th distance, so
    the tile candidates of most rows cannot be certified and the rows go
    through the batched exact recompute; forward lists and adjacency still
    match the oracle (exact ties, broken by index on both sides)."""
    if case == "wide":  # dpad = 160: the recompute's any-width path
        X = _lattice(4, 5, pad_to=160)
    elif case == "d96":  # dpad = 96: three chunks of 32 per lane
        X = _lattice(6, 4, pad_to=96)
    else:
        X = _lattice(8, 4)
    kw, okw = dict(seed=2), dict(seed=2)
    if case == "knn":
        kw["graph"], okw["graph"] = H.GRAPH_KNN, O.GRAPH_KNN
    if case == "nsw_tc":
        kw["tiles"] = H.TILES_TCGEN05
    elif case != "wide":
        kw["tiles"] = H.TILES_SIMT
    oidx = O.build_index(X, **okw)
    gidx = _gpu_index(X, **kw)
    assert gidx.info()["uncertified_rows"] > 0
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X)


@pytest.mark.parametrize("graph", ["nsw", "knn"])
def test_halving_sampler_parity(graph):
    """Layers from the halving sampler of Alg. 3 (BuildEpsNetDiscV2) are
    bit-exact against the oracle's, and the graphs built on them match."""
    X = synth.uniform_cube(6001, 24, seed=11)
    kw, okw = dict(seed=3, sampler=H.SAMPLER_HALVING), dict(seed=3, sampler=O.SAMPLER_HALVING)
    if graph == "knn":
        kw["graph"], okw["graph"] = H.GRAPH_KNN, O.GRAPH_KNN
    oidx = O.build_index(X, **okw)
    gidx = _gpu_index(X, **kw)
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X)


def test_tcgen05_tiles_reject_wide_lists():
    """The tensor-core epilogue keeps 32 candidates per row: forward lists
    of more than 16 links need the SIMT engine."""
    with pytest.raises(H.HennError) as e:
        _gpu_index(synth.uniform_cube(500, 20, seed=1), tiles=H.TILES_TCGEN05, M=24)
    assert e.value.status == 6
    assert _gpu_index(synth.uniform_cube(500, 20, seed=1), M=24).info()["tile_engine"] == H.TILES_SIMT


# ------------------------------------------------------------ search

def _recall(ids, gi, gd):
    return O.recall_at_k(ids, gi, gd).mean()


@pytest.mark.parametrize("ef", [10, 32, 64, 128])
def test_search_parity_uniform10k(uniform10k, ef):
    X, Q, oidx, gidx = uniform10k
    gi, gd = O.bruteforce(X, Q, 10)
    ids, dd, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=ef)
    ids, dd = ids.cpu().numpy(), dd.cpu().numpy()
    oi, od, _ = O.search(oidx, X, Q, k=10, ef=ef)
    rg, ro = _recall(ids, gi, gd), _recall(oi, gi, gd)
    assert abs(rg - ro) <= P.RECALL_TOL + 1e-12, (ef, rg, ro)
    assert P.returned_distance_error(X, Q, ids, dd) <= P.DIST_RTOL
    # results sorted, unique
    assert np.all(np.diff(dd, axis=1) >= 0)
    for q in range(len(Q)):
        assert len(set(ids[q].tolist())) == 10


@pytest.mark.parametrize("efu,l1,da", [(16, 0, 0), (16, 4, 0), (16, 0, 1), (32, 8, 1)])
def test_search_upper_beam_parity(uniform10k, efu, l1, da):
    """Beams on the upper layers (width ef_upper, ef_l1 on layer 1, and
    entering each layer at all candidates of the layer above)."""
    X, Q, oidx, gidx = uniform10k
    gi, gd = O.bruteforce(X, Q, 10)
    ids, dd, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=32, ef_upper=efu, ef_l1=l1, descend_all=da)
    oi, od, _ = O.search(oidx, X, Q, k=10, ef=32, ef_upper=efu, ef_l1=l1, descend_all=da)
    assert abs(_recall(ids.cpu().numpy(), gi, gd) - _recall(oi, gi, gd)) <= P.RECALL_TOL + 1e-12
    assert P.returned_distance_error(X, Q, ids.cpu().numpy(), dd.cpu().numpy()) <= P.DIST_RTOL


@pytest.mark.parametrize("efu,da", [(1, 0), (16, 0), (16, 1)])
def test_search_exact_upper_parity(uniform10k, efu, da):
    """Upper layers of at most exact_upper points give their exact candidate
    sets instead of a walk: same answers as the oracle's."""
    X, Q, oidx, gidx = uniform10k
    gi, gd = O.bruteforce(X, Q, 10)
    ids, dd, st = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=32, ef_upper=efu, descend_all=da,
                              exact_upper=64, stats=True)
    oi, od, ost = O.search(oidx, X, Q, k=10, ef=32, ef_upper=efu, descend_all=da, exact_upper=64)
    ids = ids.cpu().numpy()
    assert abs(_recall(ids, gi, gd) - _recall(oi, gi, gd)) <= P.RECALL_TOL + 1e-12
    assert P.returned_distance_error(X, Q, ids, dd.cpu().numpy()) <= P.DIST_RTOL
    assert np.mean(np.all(ids == oi, axis=1)) >= 0.98
    small = sum(int(s) for s in oidx["sizes"][1:] if s <= 64)
    assert small > 0 and np.all(st.cpu().numpy()[:, 0] >= small)


@pytest.mark.parametrize("layer", [0, 1])
def test_greedy_probe_matches_oracle(uniform10k, layer):
    """henn_greedy_probe walks the same GreedySearch (Alg. 4) as the oracle's
    on the same layer graph: from every start it stops at the same local
    minimum, with the same number of moves (FP32 against FP64 distances:
    a differing end point must be a near tie)."""
    X, Q, oidx, gidx = uniform10k
    lay = gidx.layer(layer)
    size = len(lay["adj"])
    nq, S = 40, 6
    starts = (synth.uniform_stream(5, 7, nq * S) * size).astype(np.int64).reshape(nq, S)
    starts[0, 0] = size + 3  # out of range -> -1
    node, dist, hops = gidx.greedy_probe(torch.from_numpy(Q[:nq]).to(DEV), torch.from_numpy(starts).to(DEV),
                                         layer=layer)
    node, hops = node.cpu().numpy(), hops.cpu().numpy()
    assert node[0, 0] == -1
    ids = None if layer == 0 else lay["ids"].astype(np.int64)
    same = total = 0
    for q in range(nq):
        for j in range(S):
            if q == 0 and j == 0:
                continue
            o_node, o_hops, _ = O.greedy_layer(X, ids, lay["adj"], Q[q], int(starts[q, j]))
            total += 1
            if o_node == node[q, j]:
                same += 1
                assert o_hops == hops[q, j]
            else:
                pts = X if ids is None else X[ids]
                da = float(((pts[o_node].astype(np.float64) - Q[q]) ** 2).sum())
                db = float(((pts[node[q, j]].astype(np.float64) - Q[q]) ** 2).sum())
                assert abs(da - db) <= 1e-5 * da, (q, j, da, db)
    assert same >= 0.99 * total


def test_search_host_buffers_equal_device(uniform10k):
    """The host-buffer form (copies inside the call) returns the same."""
    X, Q, oidx, gidx = uniform10k
    a_ids, a_d, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=48)
    b_ids, b_d, _ = gidx.search(Q, k=10, ef=48)
    assert np.array_equal(a_ids.cpu().numpy(), b_ids)
    assert np.array_equal(a_d.cpu().numpy(), b_d)


def test_search_uneven_k_ef(uniform10k):
    """One launch serves queries with different k and beam widths; each
    query's result equals its result in a uniform launch."""
    X, Q, oidx, gidx = uniform10k
    Qd = torch.from_numpy(Q).to(DEV)
    rng = np.random.default_rng(0)
    k = rng.choice([1, 5, 10, 37], size=len(Q)).astype(np.int32)
    ef = synth.log_uniform_int(len(Q), 16, 256, seed=3)
    ids, dd, st = gidx.search(Qd, k=torch.from_numpy(k).to(DEV), ef=torch.from_numpy(ef).to(DEV), out_stride=40,
                              stats=True)
    ids = ids.cpu().numpy()
    for q in range(0, len(Q), 50):
        one, _, _ = gidx.search(Qd[q:q + 1], k=int(k[q]), ef=int(ef[q]), keys=torch.tensor([q], dtype=torch.int64,
                                                                                            device=DEV).view(torch.int64))
        assert np.array_equal(ids[q, :k[q]], one.cpu().numpy()[0])
        assert np.all(ids[q, k[q]:] == -1)
    # oracle with the same per-query parameters
    gi, gd = O.bruteforce(X, Q, 37)
    oi, _, _ = O.search(oidx, X, Q, k=k, ef=ef, out_stride=40)
    rg_all, ro_all = [], []
    for kk in [1, 5, 10, 37]:
        sel = k == kk
        rg = O.recall_at_k(ids[sel][:, :kk], gi[sel][:, :kk], gd[sel][:, :kk])
        ro = O.recall_at_k(oi[sel][:, :kk], gi[sel][:, :kk], gd[sel][:, :kk])
        rg_all.append(rg)
        ro_all.append(ro)
        assert abs(rg.mean() - ro.mean()) <= 0.01, (kk, rg.mean(), ro.mean())  # per-k subsets of ~250 queries
    # over the whole batch: the parity tolerance
    assert abs(np.concatenate(rg_all).mean() - np.concatenate(ro_all).mean()) <= P.RECALL_TOL + 1e-12
    assert np.mean([np.array_equal(ids[q, :k[q]], oi[q, :k[q]]) for q in range(len(Q))]) >= 0.97


# Recall gap of the precision forms against the FP64 oracle on the same
# graphs, both directions.  BF16 keeps the 0.5-point parity tolerance; FP8
# E4M3 (3 fraction bits, up to 6 % per element) reorders the beam itself:
# on this 20k x 128 mixture at ef 64 it finds 4.4 points less than the
# oracle (0.922 against 0.966 on a GB300), the stated figure for that form,
# bounded here by 5 points.
PRECISION_TOL = {"bf16": P.RECALL_TOL, "fp8": 0.05}


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_search_precision_forms(storage):
    """BF16 / FP8-E4M3 traversal with exact FP32 rerank: returned distances
    are FP32-exact, recall tracks the FP64 oracle searching the same
    graphs (2,000 queries)."""
    Xs, rng_ = synth.gaussian_mixture(20000, 128, 200, seed=0, rescale_to_255=True)
    Q, _ = synth.gaussian_mixture(2000, 128, 200, seed=1, rescale_from=rng_, rescale_to_255=True)
    st = H.BF16 if storage == "bf16" else H.FP8E4M3
    gidx = _gpu_index(Xs, storage=st, seed=1)
    gi, gd = O.bruteforce(Xs, Q, 10)
    oidx = P.oracle_view(gidx, seed=1)
    ids, dd, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=64, ef_upper=16)
    oi, _, _ = O.search(oidx, Xs, Q, k=10, ef=64, ef_upper=16)
    ids, dd = ids.cpu().numpy(), dd.cpu().numpy()
    assert P.returned_distance_error(Xs, Q, ids, dd) <= P.DIST_RTOL
    rg, ro = _recall(ids, gi, gd), _recall(oi, gi, gd)
    print(f"{storage}: gpu {rg:.4f} oracle {ro:.4f}")
    assert abs(rg - ro) <= PRECISION_TOL[storage] + 1e-12, (storage, rg, ro)


def test_search_angular():
    X, _ = synth.gaussian_mixture(6000, 96, 50, seed=0, normalise=True)
    Q, _ = synth.gaussian_mixture(2000, 96, 50, seed=1, normalise=True)
    oidx = O.build_index(X, metric=O.ANGULAR, seed=8)
    gi, gd = O.bruteforce(X, Q, 10, metric=O.ANGULAR)
    oi, _, _ = O.search(oidx, X, Q, k=10, ef=64)
    for st in (H.F32, H.BF16):
        gidx = _gpu_index(X, metric=H.ANGULAR, storage=st, seed=8)
        _layers_equal(gidx, oidx)
        ids, dd, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=64)
        ids, dd = ids.cpu().numpy(), dd.cpu().numpy()
        assert P.returned_distance_error(X, Q, ids, dd, metric=1) <= P.DIST_RTOL
        rg, ro = _recall(ids, gi, gd), _recall(oi, gi, gd)
        print(f"angular storage {st}: gpu {rg:.4f} oracle {ro:.4f}")
        assert abs(rg - ro) <= P.RECALL_TOL + 1e-12, (st, rg, ro)


@pytest.mark.parametrize("lam", [4.0, 256.0])
def test_exponential_workload_parity(lam):
    """The paper's own synthetic data (App. G: i.i.d. exponential
    coordinates), d = 32: layers bit-exact, graphs within the near-tie
    rule, and the plain greedy descent of Alg. 4 with the layer-0 beam
    within 0.5 points of the oracle's recall."""
    X = synth.exponential(20000, 32, lam, seed=0)
    Q = synth.exponential(1000, 32, lam, seed=1)
    oidx = O.build_index(X, seed=0)
    gidx = _gpu_index(X, seed=0)
    _layers_equal(gidx, oidx)
    _graph_parity(gidx, oidx, X)
    gi, gd = O.bruteforce(X, Q, 10)
    for ef in (16, 64):
        ids, dd, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=ef)
        oi, _, _ = O.search(oidx, X, Q, k=10, ef=ef)
        ids, dd = ids.cpu().numpy(), dd.cpu().numpy()
        assert abs(_recall(ids, gi, gd) - _recall(oi, gi, gd)) <= P.RECALL_TOL + 1e-12, ef
        assert P.returned_distance_error(X, Q, ids, dd) <= P.DIST_RTOL
        assert np.mean(np.all(ids == oi, axis=1)) >= 0.98


# ------------------------------------------------------- edge cases

def test_edge_cases():
    # one point
    X = np.array([[1.0, 2.0, 3.0]], np.float32)
    g = _gpu_index(X)
    ids, dd, _ = g.search(np.array([[1.0, 2.0, 4.0]], np.float32), k=3, ef=5)
    assert ids.tolist() == [[0, -1, -1]] and abs(dd[0, 0] - 1.0) < 1e-6 and np.isinf(dd[0, 1])
    # fewer points than 2^m: no upper layer, k > n pads
    X = synth.uniform_cube(9, 3, seed=17)
    Q = synth.uniform_cube(5, 3, seed=18)
    g = _gpu_index(X, seed=1)
    assert g.info()["L"] == 0
    ids, dd, _ = g.search(Q, k=12, ef=20)
    gi, _ = O.bruteforce(X, Q, 9)
    assert np.array_equal(ids[:, :9], gi) and np.all(ids[:, 9:] == -1)
    # empty batch
    ids, dd, _ = g.search(np.zeros((0, 3), np.float32), k=4, ef=8)
    assert ids.shape == (0, 4)
    # invalid arguments -> HENN_ERR_INVALID_ARG, no state change
    with pytest.raises(H.HennError) as e:
        g.search(Q, k=0, ef=8)
    assert e.value.status == 1
    with pytest.raises(H.HennError) as e:
        g.search(Q, k=5, ef=5000)
    assert e.value.status == 1
    with pytest.raises(H.HennError) as e:
        _gpu_index(np.zeros((10, 2000), np.float32))
    assert e.value.status == 1
    # the index still answers
    ids2, _, _ = g.search(Q, k=3, ef=8)
    assert np.array_equal(ids2, ids[:, :3]) or ids2.shape == (5, 3)


def test_quantize_bit_exact():
    rng = np.random.default_rng(3)
    X = (rng.normal(size=(300, 77)) * np.exp(rng.normal(size=(300, 1)) * 3)).astype(np.float32)
    X[5] = 0.0
    Xd = torch.from_numpy(X).to(DEV)
    b, _ = H.quantize_rows(Xd, H.BF16)
    assert np.array_equal(b.cpu().numpy().view(np.uint16).reshape(-1), O.bf16_bits(X.reshape(-1)))
    c, s = H.quantize_rows(Xd, H.FP8E4M3)
    s = s.cpu().numpy()
    m = np.abs(X).max(1)
    want_s = np.where(m > 0, (m / np.float32(448.0)).astype(np.float32), np.float32(1.0))
    assert np.array_equal(s, want_s)
    v = (X / want_s[:, None]).astype(np.float32)
    assert np.array_equal(c.cpu().numpy().reshape(-1), O.e4m3_bits(v.reshape(-1)))


@pytest.mark.parametrize("k,metric", [(1, 0), (10, 0), (100, 0), (10, 1)])
def test_exact_knn(k, metric):
    X, _ = synth.gaussian_mixture(7000, 70, 30, seed=0, normalise=metric == 1)
    Q, _ = synth.gaussian_mixture(300, 70, 30, seed=1, normalise=metric == 1)
    ids, dd = H.exact_knn(torch.from_numpy(X).to(DEV), torch.from_numpy(Q).to(DEV), k, metric=metric)
    gi, gd = O.bruteforce(X, Q, k, metric=metric)
    ids = ids.cpu().numpy()
    assert O.recall_at_k(ids, gi, gd).mean() >= 0.9999
    assert P.returned_distance_error(X, Q, ids, dd.cpu().numpy(), metric) <= P.DIST_RTOL


# --------------------------------------------- full size, sampled checks

@pytest.fixture(scope="module")
def mixture1m():
    X, Q, info = synth.workload("mixture-1m-d128")
    gidx = _gpu_index(X, seed=0)
    return X, Q, gidx


def test_full_size_layers_bit_exact(mixture1m):
    """1M x 128 (the benchmarked workload): membership of every layer."""
    X, Q, gidx = mixture1m
    oidx = O.build_layers(X, seed=0)
    _layers_equal(gidx, oidx)


def test_full_size_sampled_forward_rows(mixture1m):
    """Forward lists of 64 sampled rows per layer, computed one by one."""
    X, Q, gidx = mixture1m
    info = gidx.info()
    rng = np.random.default_rng(11)
    total = ex_total = 0
    for i in range(info["L"] + 1):
        lay = gidx.layer(i)
        ids = np.arange(info["sizes"][0]) if i == 0 else lay["ids"].astype(np.int64)
        rows = rng.choice(len(ids), size=min(64, len(ids)), replace=False)
        orc = np.stack([O.forward_row(X, ids, 0, i, int(p), M=16)[0] for p in rows])
        for r_i, p in enumerate(rows):
            e, ex, un, _ = _row_compare_fullsize(lay["fwd"][p], orc[r_i], X, ids, p)
            assert un == 0, (i, p)
            total += e
            ex_total += ex
    assert ex_total <= max(1, P.EXCUSED_BUDGET * total)


def _row_compare_fullsize(g_row, o_row, X, ids, p):
    g = set(int(v) for v in g_row if v >= 0)
    o = set(int(v) for v in o_row if v >= 0)
    edges = len(o)
    if g == o:
        return edges, 0, 0, None
    _, ex, un, _ = P._row_rule(g, o, X, ids, p, 0)
    return edges, ex, un, None
