"""Serving benchmark: open-loop request stream against henn_serve_*.

Requests arrive as a Poisson process; each carries a batch of queries
(size log-uniform in [1, max_batch]), k uniform in {10, 100} and a beam
width log-uniform in [64, 512].  A submitter thread submits at the arrival
times (a request refused for lack of ring rows or slots is retried; the
wait counts in its latency), a poller thread collects finished requests.
Latency = collection time - arrival time.  Prints one JSON line per offered
rate with p50 / p99 latency (ms) and the achieved query throughput.

    python -m paper_2505_17368_gb300.serve_bench --workload mixture-1m-d128 --rates 2e5,1e6,3e6
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run_rate(srv, Q, rate_qps, seconds, max_batch, seed):
    rng = np.random.default_rng(seed)
    mean_batch = (max_batch - 1) / math.log(max_batch)  # mean of log-uniform [1, max_batch]
    req_rate = rate_qps / mean_batch
    reqs = []
    t = 0.0
    while t < seconds:
        t += rng.exponential(1.0 / req_rate)
        b = int(min(max_batch, max(1, round(math.exp(rng.uniform(0, math.log(max_batch)))))))
        k = int(rng.choice([10, 100]))
        ef = int(round(math.exp(rng.uniform(math.log(64), math.log(512)))))
        reqs.append((t, b, k, ef))
    pending = []
    lock = threading.Lock()
    lat = []
    done_q = [0]
    stop = threading.Event()
    t0 = time.perf_counter()

    def submitter():
        off = 0
        for (ta, b, k, ef) in reqs:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            if off + b > len(Q):
                off = 0
            while True:
                rid = srv.submit(Q[off:off + b], k=k, ef=ef)
                if rid is not None:
                    break
                time.sleep(50e-6)
            with lock:
                pending.append((rid, ta, b))
            off += b
        stop.set()

    def poller():
        while True:
            with lock:
                cur = list(pending)
            if not cur and stop.is_set():
                return
            for item in cur:
                rid, ta, b = item
                r = srv.poll(rid)
                if r is not None:
                    lat.append(time.perf_counter() - t0 - ta)
                    done_q[0] += b
                    with lock:
                        pending.remove(item)
            time.sleep(20e-6)

    th = [threading.Thread(target=submitter), threading.Thread(target=poller)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    elapsed = time.perf_counter() - t0
    lat_ms = np.array(lat) * 1e3
    return {
        "offered_qps": rate_qps, "achieved_qps": done_q[0] / elapsed, "requests": len(lat),
        "queries": done_q[0], "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
        "seconds": elapsed,
    }


def batched_same_mix(idx, Q, seconds, max_batch, seed, ef_upper, descend_all, ef_l1, exact_upper, exact_method,
                     gt=None):
    """The batched ceiling for the same query mix: the queries of the same
    generated request stream (batch sizes, k, ef) answered by henn_search
    calls over batches of 10,000 queries with per-query k and ef (no
    arrivals, no admission); (queries per second of device time, mean
    recall@k against gt's exact neighbours, or None)."""
    import torch

    rng = np.random.default_rng(seed)
    ks, efs = [], []
    while len(ks) < 10000:
        b = int(min(max_batch, max(1, round(math.exp(rng.uniform(0, math.log(max_batch)))))))
        k = int(rng.choice([10, 100]))
        ef = int(round(math.exp(rng.uniform(math.log(64), math.log(512)))))
        ks += [k] * b
        efs += [ef] * b
    n = min(10000, len(Q))
    kq = torch.tensor(ks[:n], dtype=torch.int32, device="cuda")
    eq = torch.tensor(efs[:n], dtype=torch.int32, device="cuda")
    Qd = torch.from_numpy(np.ascontiguousarray(Q[:n])).cuda()
    kw = dict(k=kq, ef=eq, out_stride=100, ef_upper=ef_upper, descend_all=descend_all, ef_l1=ef_l1,
              exact_upper=exact_upper, exact_method=exact_method)
    idx.search(Qd, **kw)
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        idx.search(Qd, **kw)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    rec = None
    if gt is not None:
        ids = idx.search(Qd, **kw)[0].cpu().numpy()
        kk = np.array(ks[:n])
        rec = float(np.mean([len(set(ids[q, :kk[q]].tolist()) & set(gt[q, :kk[q]].tolist())) / kk[q]
                             for q in range(n)]))
    return n / float(np.median(ts)), rec


def main():
    import torch

    import paper_2505_17368_gb300 as H
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="mixture-1m-d128")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--rates", default="2e5,1e6,2e6,4e6")
    ap.add_argument("--seconds", type=float, default=3.0)
    ap.add_argument("--max-batch", type=int, default=4096)
    ap.add_argument("--ef-upper", type=int, default=64)
    ap.add_argument("--descend-all", type=int, default=0)
    ap.add_argument("--ef-l1", type=int, default=0)
    ap.add_argument("--exact-upper", default="0", help="exact layer size bound, or L<i> for the size of layer i")
    ap.add_argument("--tiles", type=int, default=0)
    args = ap.parse_args()
    X, Q, info = synth.workload(args.workload, n=args.n, nq=20000)
    metric = H.ANGULAR if info["metric"] == "angular" else H.L2
    t = time.perf_counter()
    idx = H.Index(torch.from_numpy(X).cuda(), metric=metric, storage=H.BF16, seed=0, tiles=args.tiles)
    build_s = time.perf_counter() - t
    sizes = idx.info()["sizes"]
    xu = args.exact_upper
    xu = (sizes[int(xu[1:])] if int(xu[1:]) < len(sizes) else 0) if xu.startswith("L") else int(xu)
    beam = dict(ef_upper=args.ef_upper, descend_all=args.descend_all, ef_l1=args.ef_l1, exact_upper=xu)
    # exact neighbours (FP32, on the device) of the first 10,000 queries, for the recall of the mix
    Xd = torch.from_numpy(X).cuda()
    gt = H.exact_knn(Xd, torch.from_numpy(np.ascontiguousarray(Q[:10000])).cuda(), 100, metric=metric)[0].cpu().numpy()
    del Xd
    ceiling = {}
    for m in ([H.EXACT_SORT, H.EXACT_TILES] if xu else [H.EXACT_SORT]):
        try:
            qps, rec = batched_same_mix(idx, Q, args.seconds, args.max_batch, 99, exact_method=m, gt=gt, **beam)
            ceiling["tiles" if m == H.EXACT_TILES else "sort"] = {"qps": qps, "recall_at_k": rec}
        except H.HennError as e:  # e.g. a layer too large for the in-kernel sort of a batched call
            ceiling["tiles" if m == H.EXACT_TILES else "sort"] = str(e)
    print(json.dumps({"workload": args.workload, "n": len(X), "layers": sizes, **beam,
                      "batched_same_mix": ceiling}), flush=True)
    srv = H.Server(idx, ring_rows=1 << 17, max_requests=4096, max_k=100, max_ef=512, **beam)
    for r in [float(v) for v in args.rates.split(",")]:
        res = run_rate(srv, Q, r, args.seconds, args.max_batch, seed=int(r) % 1000)
        res.update(workload=args.workload, n=len(X), build_seconds=build_s, form="bf16 + fp32 rerank", **beam)
        print(json.dumps(res), flush=True)
    srv.close()


if __name__ == "__main__":
    main()
