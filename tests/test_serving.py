"""Continuous batching (henn_serve_*): requests that arrive while others are
on the GPU are admitted as ring rows and slots free up, run concurrently in
one persistent kernel, and each request's results are the same alone and in
the mix (bitwise: a query's result depends only on the query, k, ef and
its entry key)."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_17368_gb300 as H  # noqa: E402


def _wait(srv, rid, timeout=60.0):
    t0 = time.time()
    while True:
        r = srv.poll(rid)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(0.0005)


def _data():
    X, rng = synth.gaussian_mixture(20000, 64, 100, seed=0, rescale_to_255=True)
    Q, _ = synth.gaussian_mixture(3000, 64, 100, seed=1, rescale_from=rng, rescale_to_255=True)
    return X, Q


@pytest.fixture(scope="module")
def index_and_queries():
    X, Q = _data()
    idx = H.Index(torch.from_numpy(X).cuda(), storage=H.BF16, seed=3)
    return idx, Q


def _requests(nq_total, seed):
    rng = np.random.default_rng(seed)
    reqs, at = [], 0
    while at < nq_total:
        b = int(min(nq_total - at, np.exp(rng.uniform(0, np.log(400)))))
        k = int(rng.choice([10, 100]))
        ef = int(np.exp(rng.uniform(np.log(64), np.log(512))))
        reqs.append((at, b, k, ef))
        at += b
    return reqs


def test_alone_equals_in_mix(index_and_queries):
    idx, Q = index_and_queries
    reqs = _requests(len(Q), 0)
    srv = H.Server(idx, ring_rows=2048, max_requests=16, max_k=100, max_ef=512, ef_upper=16)
    results = {}
    errors = []

    def client(part):
        # submit as the budget allows; while refused, collect finished
        # requests (ring rows are released only when a request is collected)
        try:
            outstanding = []
            for (at, b, k, ef) in part:
                keys = np.arange(at, at + b, dtype=np.uint64)
                while True:
                    rid = srv.submit(Q[at:at + b], k=k, ef=ef, keys=keys)
                    if rid is not None:
                        break
                    for item in list(outstanding):
                        r = srv.poll(item[0])
                        if r is not None:
                            results[item[1]] = item[2:] + r
                            outstanding.remove(item)
                    time.sleep(0.0002)
                outstanding.append((rid, at, b, k, ef))
            for rid, at, b, k, ef in outstanding:
                results[at] = (b, k, ef) + _wait(srv, rid)
        except Exception as e:  # pragma: no cover
            errors.append(e)

    th = [threading.Thread(target=client, args=(reqs[i::4],)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    srv.close()
    # every request alone, through the batch API with the same keys
    for at, b, k, ef in reqs:
        _, _, _, ids_mix, d_mix = results[at]
        keys = torch.arange(at, at + b, dtype=torch.int64, device="cuda")
        ids, dd, _ = idx.search(torch.from_numpy(Q[at:at + b]).cuda(), k=k, ef=ef, ef_upper=16, keys=keys)
        assert np.array_equal(ids.cpu().numpy(), ids_mix), at
        assert np.array_equal(dd.cpu().numpy(), d_mix), at
    # and alone in a fresh server
    srv2 = H.Server(idx, ring_rows=2048, max_requests=4, max_k=100, max_ef=512, ef_upper=16)
    for at, b, k, ef in reqs[:5]:
        rid = srv2.submit(Q[at:at + b], k=k, ef=ef, keys=np.arange(at, at + b, dtype=np.uint64))
        ids, dd = _wait(srv2, rid)
        assert np.array_equal(ids, results[at][3]) and np.array_equal(dd, results[at][4])
    srv2.close()


def test_served_results_track_oracle(index_and_queries):
    """A mixed stream (batch sizes log-uniform, k in {10, 100}, ef
    log-uniform in [64, 512]) through the server against the FP64 oracle
    searching the same GPU-built graphs with each query's own k, ef and
    entry key: recall@k against FP64 brute force within the parity
    tolerance over the stream, returned distances within 1e-4 of FP64."""
    import oracle as O
    from tests import parity as P

    idx, Q = index_and_queries
    X, _ = _data()
    view = P.oracle_view(idx, seed=3)
    reqs = _requests(len(Q), 7)
    srv = H.Server(idx, ring_rows=4096, max_requests=32, max_k=100, max_ef=512, ef_upper=16)
    pending, served = [], {}
    for at, b, k, ef in reqs:
        keys = np.arange(at, at + b, dtype=np.uint64) * 7 + 1
        while (rid := srv.submit(Q[at:at + b], k=k, ef=ef, keys=keys)) is None:
            for item in list(pending):
                r = srv.poll(item[0])
                if r is not None:
                    served[item[1]] = r
                    pending.remove(item)
        pending.append((rid, at))
    for rid, at in pending:
        served[at] = _wait(srv, rid)
    srv.close()
    gi, gd = O.bruteforce(X, Q, 100)
    rg, ro = [], []
    for at, b, k, ef in reqs:
        ids, dd = served[at]
        keys = np.arange(at, at + b, dtype=np.uint64) * 7 + 1
        oi, _, _ = O.search(view, X, Q[at:at + b], k=k, ef=ef, ef_upper=16, keys=keys)
        rg.append(O.recall_at_k(ids, gi[at:at + b, :k], gd[at:at + b, :k]))
        ro.append(O.recall_at_k(oi, gi[at:at + b, :k], gd[at:at + b, :k]))
        assert P.returned_distance_error(X, Q[at:at + b], ids, dd) <= P.DIST_RTOL
    rg, ro = np.concatenate(rg).mean(), np.concatenate(ro).mean()
    print(f"served {rg:.4f} oracle {ro:.4f}")
    assert abs(rg - ro) <= P.RECALL_TOL + 1e-12, (rg, ro)


def test_exact_layer_and_seeded_beams_in_serving(index_and_queries):
    """A server may take an upper layer's exact candidate set (in-kernel
    sort) and seed narrower beams below it (descend_all, ef_l1): each
    request's results equal henn_search's with the same options."""
    idx, Q = index_and_queries
    sizes = idx.info()["sizes"]
    xu = sizes[2]
    kw = dict(ef_upper=16, descend_all=1, ef_l1=8, exact_upper=xu)
    srv = H.Server(idx, ring_rows=4096, max_requests=8, max_k=100, max_ef=512, **kw)
    for at, b, k, ef in _requests(600, 11)[:12]:
        keys = np.arange(at, at + b, dtype=np.uint64)
        rid = srv.submit(Q[at:at + b], k=k, ef=ef, keys=keys)
        assert rid is not None
        ids_s, d_s = _wait(srv, rid)
        ids, dd, _ = idx.search(torch.from_numpy(Q[at:at + b]).cuda(), k=k, ef=ef, keys=torch.from_numpy(
            keys.astype(np.int64)).cuda(), exact_method=H.EXACT_SORT, **kw)
        assert np.array_equal(ids.cpu().numpy(), ids_s) and np.array_equal(dd.cpu().numpy(), d_s), at
    srv.close()
    with pytest.raises(H.HennError) as e:
        H.Server(idx, ef_l1=5000)
    assert e.value.status == 1


def test_admission_budget_and_errors(index_and_queries):
    idx, Q = index_and_queries
    srv = H.Server(idx, ring_rows=100, max_requests=2, max_k=10, max_ef=128)
    with pytest.raises(H.HennError) as e:
        srv.submit(Q[:101], k=10, ef=64)
    assert e.value.status == 1
    with pytest.raises(H.HennError) as e:
        srv.submit(Q[:5], k=11, ef=64)
    assert e.value.status == 1
    with pytest.raises(H.HennError) as e:
        srv.submit(Q[:5], k=10, ef=129)
    assert e.value.status == 1
    a = srv.submit(Q[:60], k=10, ef=64)
    assert a is not None
    assert srv.submit(Q[60:120], k=10, ef=64) is None  # ring rows: 60 + 60 > 100
    b = srv.submit(Q[60:80], k=10, ef=64)
    assert b is not None
    assert srv.submit(Q[80:81], k=10, ef=64) is None  # both request slots in use
    _wait(srv, a)
    c = srv.submit(Q[80:120], k=10, ef=64)  # rows of a released
    assert c is not None
    _wait(srv, b)
    _wait(srv, c)
    with pytest.raises(H.HennError):
        srv.poll(c)  # already collected
    srv.close()


def test_idle_exit_and_relaunch(index_and_queries):
    idx, Q = index_and_queries
    srv = H.Server(idx, ring_rows=512, max_requests=8, max_k=10, max_ef=128, idle_ms=2)
    r1 = srv.submit(Q[:50], k=10, ef=64)
    ids1, _ = _wait(srv, r1)
    time.sleep(0.1)  # the kernel has left by now
    r2 = srv.submit(Q[:50], k=10, ef=64, keys=(np.uint64(r1) << np.uint64(20)) + np.arange(50, dtype=np.uint64))
    ids2, _ = _wait(srv, r2)
    assert np.array_equal(ids1, ids2)
    srv.close()


def test_destroy_with_requests_in_flight(index_and_queries):
    idx, Q = index_and_queries
    srv = H.Server(idx, ring_rows=4096, max_requests=8, max_k=10, max_ef=512)
    for i in range(4):
        srv.submit(Q[i * 500:(i + 1) * 500], k=10, ef=512)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30
