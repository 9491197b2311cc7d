"""The exact upper layer (the nearest points of the lowest layer with at most
exact_upper points, then the walk below it) found three ways through the C
ABI: sorted in the visited table (EXACT_SORT), from batched distance tiles
with a certified rescore (EXACT_TILES: tcgen05 tiles of 128 x 256 or
128 x 128, the row block streamed for rows wider than 128 values),
and by a scan of the layer (EXACT_SCAN).  The three give the same set, so
the same answers bit for bit; the answers track the FP64 oracle's exact
layer.  Tolerances: tests/parity.py.
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
METHODS = (H.EXACT_SORT, H.EXACT_TILES, H.EXACT_SCAN)


def _gpu_index(X, **kw):
    return H.Index(torch.from_numpy(np.ascontiguousarray(X)).to(DEV), **kw)


def _exact_layer(sizes, xu):
    return next(i for i in range(1, len(sizes)) if sizes[i] <= xu)


def _run(gidx, Q, methods=METHODS, **kw):
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(DEV)
    out = {}
    for m in methods:
        ids, dd, st = gidx.search(Qd, exact_method=m, stats=True, **kw)
        out[m] = (ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy())
    return out


def _same(out):
    base = out[METHODS[0]] if METHODS[0] in out else next(iter(out.values()))
    for m, (ids, dd, _) in out.items():
        assert np.array_equal(ids, base[0]), m
        assert np.array_equal(dd, base[1]), m


@pytest.fixture(scope="module")
def uniform10k():
    X, Q, _ = synth.workload("uniform-10k-d32")
    oidx = O.build_index(X, seed=0)
    gidx = _gpu_index(X, seed=0)
    return X, Q, oidx, gidx


@pytest.mark.parametrize("xu,efu,da", [(1000, 1, 0), (1000, 16, 0), (1000, 16, 1), (1000, 32, 1), (64, 8, 1),
                                       (10**9, 1, 0)])
def test_methods_identical_and_track_oracle(uniform10k, xu, efu, da):
    X, Q, oidx, gidx = uniform10k
    sizes = gidx.info()["sizes"]
    li = _exact_layer(sizes, xu)
    # one visited-table size for every method, large enough for SORT
    out = _run(gidx, Q, k=10, ef=32, ef_upper=efu, descend_all=da, exact_upper=xu, hash_bits=12)
    _same(out)
    ids, dd, _ = out[H.EXACT_TILES]
    gi, gd = O.bruteforce(X, Q, 10)
    oi, _, _ = O.search(oidx, X, Q, k=10, ef=32, ef_upper=efu, descend_all=da, exact_upper=xu)
    rg, ro = O.recall_at_k(ids, gi, gd).mean(), O.recall_at_k(oi, gi, gd).mean()
    assert abs(rg - ro) <= P.RECALL_TOL + 1e-12, (rg, ro)
    assert P.returned_distance_error(X, Q, ids, dd) <= P.DIST_RTOL
    assert np.mean(np.all(ids == oi, axis=1)) >= 0.98
    # the scan evaluates the whole layer; the certified tiles rescore 32
    # candidates for nearly every query, unless all 32 seed the next layer
    # (the 32nd rescored distance cannot be certified against the 32nd tile
    # distance: those queries scan)
    st_scan, st_tiles = out[H.EXACT_SCAN][2], out[H.EXACT_TILES][2]
    assert np.all(st_scan[:, 0] >= sizes[li])
    if sizes[li] > 64 and not (da and efu >= 32):
        assert st_tiles[:, 0].sum() < st_scan[:, 0].sum()


@pytest.mark.parametrize("case", ["bf16-d128", "fp8-d128", "angular-bf16-d96", "f32-d200"])
def test_tiles_equal_scan(case):
    """Storage forms, the angular metric and rows wider than 128 values
    (streamed tensor-core tiles): the certified tile candidates give the
    scan's set."""
    rng_seed = {"bf16-d128": 3, "fp8-d128": 4, "angular-bf16-d96": 5, "f32-d200": 6}[case]
    if case.startswith("angular"):
        X, _ = synth.gaussian_mixture(30000, 96, 100, seed=rng_seed, normalise=True)
        Q, _ = synth.gaussian_mixture(2000, 96, 100, seed=rng_seed + 100, normalise=True)
        kw = dict(metric=H.ANGULAR, storage=H.BF16)
    elif case.startswith("f32-d200"):
        X, r = synth.gaussian_mixture(20000, 200, 100, seed=rng_seed, rescale_to_255=True)
        Q, _ = synth.gaussian_mixture(1000, 200, 100, seed=rng_seed + 100, rescale_from=r, rescale_to_255=True)
        kw = dict(storage=H.F32)
    else:
        X, r = synth.gaussian_mixture(40000, 128, 200, seed=rng_seed, rescale_to_255=True)
        Q, _ = synth.gaussian_mixture(2000, 128, 200, seed=rng_seed + 100, rescale_from=r, rescale_to_255=True)
        kw = dict(storage=H.BF16 if case.startswith("bf16") else H.FP8E4M3)
    gidx = _gpu_index(X, seed=2, **kw)
    sizes = gidx.info()["sizes"]
    assert len(sizes) >= 3, sizes
    for xu, efu, da in [(sizes[1], 16, 0), (sizes[1], 32, 1), (sizes[2], 16, 1)]:
        out = _run(gidx, Q, methods=(H.EXACT_TILES, H.EXACT_SCAN), k=10, ef=48, ef_upper=efu, descend_all=da,
                   exact_upper=xu)
        _same(out)
        if efu < 32:
            assert out[H.EXACT_TILES][2][:, 0].sum() < out[H.EXACT_SCAN][2][:, 0].sum()
    gi, gd = O.bruteforce(X, Q[:300], 10, metric=O.ANGULAR if case.startswith("angular") else O.L2)
    ids = out[H.EXACT_TILES][0][:300]
    assert O.recall_at_k(ids, gi, gd).mean() >= 0.8


def test_width_limit_and_timing(uniform10k):
    X, Q, oidx, gidx = uniform10k
    Qd = torch.from_numpy(Q).to(DEV)
    # descend_all seeds the next layer with the whole set: at most 32 here
    with pytest.raises(H.HennError) as e:
        gidx.search(Qd, k=10, ef=32, ef_upper=64, descend_all=1, exact_upper=1000, exact_method=H.EXACT_TILES)
    assert e.value.status == 1
    with pytest.raises(H.HennError) as e:
        gidx.search(Qd, k=10, ef=32, exact_upper=1000, exact_method=3)
    assert e.value.status == 1
    # SORT keeps its visited-table limit: the exact layer of 610 points
    # needs 2^11 slots
    with pytest.raises(H.HennError) as e:
        gidx.search(Qd, k=10, ef=32, exact_upper=1000, exact_method=H.EXACT_SORT, hash_bits=10)
    assert e.value.status == 1
    # device time of the search launches, and the launch count
    gidx.search(Qd, k=10, ef=32, exact_upper=1000, exact_method=H.EXACT_TILES, time_kernel=True)
    ms, n = gidx.last_search_ms()
    assert ms > 0 and n == 4  # query preparation, distance tiles, top-32 selection, search
    gidx.search(Qd, k=10, ef=32, time_kernel=True)
    ms, n = gidx.last_search_ms()
    assert ms > 0 and n == 1


def test_host_buffers_and_small_batches(uniform10k):
    """The host-buffer form and batches smaller than one tile row block."""
    X, Q, oidx, gidx = uniform10k
    a, ad, _ = gidx.search(torch.from_numpy(Q).to(DEV), k=10, ef=32, exact_upper=1000, exact_method=H.EXACT_TILES)
    b, bd, _ = gidx.search(Q, k=10, ef=32, exact_upper=1000, exact_method=H.EXACT_TILES)
    assert np.array_equal(a.cpu().numpy(), b) and np.array_equal(ad.cpu().numpy(), bd)
    for nq in (1, 7, 129):
        c, cd, _ = gidx.search(Q[:nq], k=10, ef=32, exact_upper=1000, exact_method=H.EXACT_TILES)
        assert np.array_equal(c, b[:nq]) and np.array_equal(cd, bd[:nq])
    # page-locked queries and results are used in place by the kernels;
    # page-locked queries with pageable results: the results are staged
    Qh = torch.from_numpy(Q).pin_memory()
    f, fd, _ = gidx.search(Qh.numpy(), k=10, ef=32, exact_upper=1000, exact_method=H.EXACT_TILES)
    assert np.array_equal(f, b) and np.array_equal(fd, bd)
    # results written into the caller's page-locked buffers, twice in a row
    ids_h = torch.full((Q.shape[0], 10), -7, dtype=torch.int64).pin_memory()
    d_h = torch.full((Q.shape[0], 10), -7.0, dtype=torch.float32).pin_memory()
    for _ in range(2):
        e, ed, _ = gidx.search(Qh.numpy(), k=10, ef=32, exact_upper=1000, exact_method=H.EXACT_TILES,
                               out=(ids_h.numpy(), d_h.numpy()))
        assert np.array_equal(ids_h.numpy(), b) and np.array_equal(d_h.numpy(), bd)
        assert np.shares_memory(e, ids_h.numpy()) and np.shares_memory(ed, d_h.numpy())
    with pytest.raises(H.HennError):
        gidx.search(Q, k=10, ef=32, out=(np.empty((Q.shape[0], 9), np.int64), np.empty((Q.shape[0], 9), np.float32)))


def test_after_insert(uniform10k):
    """Insertions grow the upper layers: the tile operands are remade."""
    X, Q, _, _ = uniform10k
    g = _gpu_index(X[:8000], seed=0)
    assert g.info()["sizes"][1] <= 700
    g.search(Q, k=10, ef=32, exact_upper=700, exact_method=H.EXACT_TILES)
    g.insert(X[8000:])
    assert g.info()["sizes"][1] <= 700
    out = _run(g, Q, methods=(H.EXACT_TILES, H.EXACT_SCAN), k=10, ef=32, exact_upper=700)
    _same(out)


def test_full_size_tiles_equal_scan():
    """1M x 128 BF16 (the benchmarked workload): the exact layer of 3,677
    points from the tcgen05 tiles equals the scan's for all 10,000 queries,
    and the benchmarked beam keeps recall@10 >= 0.95 on sampled queries."""
    X, Q, _ = synth.workload("mixture-1m-d128")
    gidx = _gpu_index(X, storage=H.BF16, seed=0)
    sizes = gidx.info()["sizes"]
    xu = sizes[2]
    out = _run(gidx, Q, methods=(H.EXACT_TILES, H.EXACT_SCAN), k=10, ef=64, ef_upper=64, exact_upper=xu)
    _same(out)
    sel = np.random.default_rng(13).choice(len(Q), 300, replace=False)
    gi, gd = O.bruteforce(X, Q[sel], 10)
    assert O.recall_at_k(out[H.EXACT_TILES][0][sel], gi, gd).mean() >= 0.95
    # a batch whose distance matrix exceeds 1 GiB goes through it in chunks
    _, Qb, _ = synth.workload("mixture-1m-d128", nq=100_000)
    outb = _run(gidx, Qb, methods=(H.EXACT_TILES, H.EXACT_SCAN), k=10, ef=48, ef_upper=16, descend_all=1,
                exact_upper=xu)
    _same(outb)
    # layer 1 (60,577 points): the running lists inside the tile epilogue
    out = _run(gidx, Q[:2000], methods=(H.EXACT_TILES, H.EXACT_SCAN), k=10, ef=48, exact_upper=sizes[1])
    _same(out)
    assert out[H.EXACT_TILES][2][:, 0].sum() < out[H.EXACT_SCAN][2][:, 0].sum()


@pytest.mark.parametrize("d", [32, 200])
def test_tile_widths_give_identical_results(d):
    """The tile's width (128 or 256 columns) changes how columns are grouped,
    not how any tile value is summed: the candidates, the certificate and the
    answers (and the per-query counters) are the same bit for bit."""
    if d == 32:
        X, Q, _ = synth.workload("uniform-10k-d32")
        Q = Q[:600]
    else:
        X, r = synth.gaussian_mixture(20000, d, 100, seed=6, rescale_to_255=True)
        Q, _ = synth.gaussian_mixture(600, d, 100, seed=106, rescale_from=r, rescale_to_255=True)
    gidx = _gpu_index(X, seed=2, storage=H.BF16)
    sizes = gidx.info()["sizes"]
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(DEV)
    for xu, efu, da in [(sizes[1], 16, 1), (sizes[2], 8, 1)]:
        res = [[t.cpu().numpy() for t in gidx.search(Qd, k=10, ef=48, ef_upper=efu, descend_all=da, exact_upper=xu,
                                                     exact_method=H.EXACT_TILES, stats=True, tile_n=n)]
               for n in (256, 128)]
        for a, b in zip(*res):
            assert np.array_equal(a, b), (d, xu)


def test_tied_distances_equal_scan():
    """Binary rows of 8 values (squared distances are the integers 0..8, and
    every vector recurs about 500 times): on the 7,578-point layer 1 most
    queries have more than 256 entries at or below the 32nd smallest chunk
    minimum, or more than 128 chunks under it, so the top-32 selection takes
    its long-list path for them and the one-round-trip path for the rest;
    the exact sets, ties ordered by index, still equal the scan's.  With one
    seed (ef_upper 1) the certificate holds for most queries (30 or so copies
    at distance 0, the 32nd candidate at 1), so the selected candidates are
    the ones the walk uses."""
    rng = np.random.default_rng(21)
    X = rng.integers(0, 2, size=(125000, 8)).astype(np.float32)
    Q = rng.integers(0, 2, size=(1000, 8)).astype(np.float32)
    for storage in (H.F32, H.BF16):
        gidx = _gpu_index(X, seed=4, storage=storage)
        sizes = gidx.info()["sizes"]
        assert len(sizes) >= 3 and sizes[1] > 4096, sizes
        for xu, efu, da in [(sizes[1], 1, 0), (sizes[1], 8, 1), (sizes[2], 16, 1)]:
            out = _run(gidx, Q, methods=(H.EXACT_TILES, H.EXACT_SCAN), k=10, ef=48, ef_upper=efu, descend_all=da,
                       exact_upper=xu)
            _same(out)
            if efu == 1:
                # most queries kept the certified candidates (fewer evaluations than a scan)
                assert out[H.EXACT_TILES][2][:, 0].sum() < out[H.EXACT_SCAN][2][:, 0].sum()


@pytest.mark.parametrize("case", ["angular-bf16-d96", "f32-d200", "per-query-k-ef"])
def test_page_locked_host_buffers_equal_device(case):
    """Queries and results in page-locked host memory are read and written in
    place by the kernels (the query preparation leaving a device copy for
    the search kernel): the same answers and counters as device-resident
    queries, for the angular metric (normalised from the staged row), rows
    wider than 128 values, and per-query k / ef (those arrays staged)."""
    if case == "angular-bf16-d96":
        X, _ = synth.gaussian_mixture(20000, 96, 100, seed=7, normalise=True)
        Q, _ = synth.gaussian_mixture(1000, 96, 100, seed=107, normalise=True)
        kw = dict(metric=H.ANGULAR, storage=H.BF16)
    elif case == "f32-d200":
        X, r = synth.gaussian_mixture(10000, 200, 100, seed=8, rescale_to_255=True)
        Q, _ = synth.gaussian_mixture(700, 200, 100, seed=108, rescale_from=r, rescale_to_255=True)
        kw = dict(storage=H.F32)
    else:
        X, r = synth.gaussian_mixture(20000, 128, 100, seed=9, rescale_to_255=True)
        Q, _ = synth.gaussian_mixture(1000, 128, 100, seed=109, rescale_from=r, rescale_to_255=True)
        kw = dict(storage=H.BF16)
    Q = np.ascontiguousarray(Q)
    gidx = _gpu_index(X, seed=3, **kw)
    sizes = gidx.info()["sizes"]
    sk = dict(ef_upper=16, descend_all=1, exact_upper=sizes[2] if len(sizes) > 2 else sizes[1],
              exact_method=H.EXACT_TILES)
    nq = len(Q)
    if case == "per-query-k-ef":
        rng = np.random.default_rng(3)
        k = rng.choice([1, 10, 32], nq).astype(np.int32)
        ef = rng.integers(16, 96, nq).astype(np.int32)
        stride = 32
        kd, efd = torch.from_numpy(k).to(DEV), torch.from_numpy(ef).to(DEV)
    else:
        k, ef, stride = 10, 48, 10
        kd, efd = k, ef
    a_ids, a_d, a_st = gidx.search(torch.from_numpy(Q).to(DEV), k=kd, ef=efd, out_stride=stride, stats=True, **sk)
    Qh = torch.from_numpy(Q).pin_memory()
    ids_h = torch.empty((nq, stride), dtype=torch.int64).pin_memory()
    d_h = torch.empty((nq, stride), dtype=torch.float32).pin_memory()
    b_ids, b_d, b_st = gidx.search(Qh.numpy(), k=k, ef=ef, out_stride=stride, stats=True,
                                   out=(ids_h.numpy(), d_h.numpy()), **sk)
    assert np.array_equal(a_ids.cpu().numpy(), b_ids) and np.array_equal(a_d.cpu().numpy(), b_d)
    assert np.array_equal(a_st.cpu().numpy(), b_st)
