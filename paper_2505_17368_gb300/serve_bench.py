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
    ap.add_argument("--tiles", type=int, default=0)
    args = ap.parse_args()
    X, Q, info = synth.workload(args.workload, n=args.n, nq=20000)
    metric = H.ANGULAR if info["metric"] == "angular" else H.L2
    t = time.perf_counter()
    idx = H.Index(torch.from_numpy(X).cuda(), metric=metric, storage=H.BF16, seed=0, tiles=args.tiles)
    build_s = time.perf_counter() - t
    srv = H.Server(idx, ring_rows=1 << 17, max_requests=4096, max_k=100, max_ef=512, ef_upper=args.ef_upper)
    for r in [float(v) for v in args.rates.split(",")]:
        res = run_rate(srv, Q, r, args.seconds, args.max_batch, seed=int(r) % 1000)
        res.update(workload=args.workload, n=len(X), build_seconds=build_s, form="bf16 + fp32 rerank",
                   ef_upper=args.ef_upper)
        print(json.dumps(res), flush=True)
    srv.close()


if __name__ == "__main__":
    main()
