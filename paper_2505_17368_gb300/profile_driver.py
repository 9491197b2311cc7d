"""Small, fixed workloads for profiling the kernels under ncu.

    python -m paper_2505_17368_gb300.profile_driver search [--n 1000000] [--nq 10000] [--ef 64] [--ef-upper 64]
                                                          [--descend-all 0] [--ef-l1 0] [--exact-upper 0]
                                                          [--exact-method 0] [--rerank-mult 4]
    python -m paper_2505_17368_gb300.profile_driver tiles  [--n 200000] [--d 128|960]

`search` builds a BF16 index of the n-point prefix of the 1M x 128 mixture
workload and runs three batched searches (profile the third launch of
k_search; with --exact-method 1 each search is a query-preparation launch,
a k_tile_topk_tc launch (after the five of the build) and k_search); `tiles` builds an index with the tcgen05 tile engine (the first
k_tile_topk_tc launch is layer 0) on the n-point prefix of the 1M x 128
mixture, or with --d 960 of the 1M x 960 one (rows streamed through the
tile pipeline).  Both print a one-line summary.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import paper_2505_17368_gb300 as H
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["search", "tiles"])
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--ef", type=int, default=64)
    ap.add_argument("--ef-upper", type=int, default=64)
    ap.add_argument("--descend-all", type=int, default=0)
    ap.add_argument("--ef-l1", type=int, default=0)
    ap.add_argument("--exact-upper", type=int, default=0)
    ap.add_argument("--exact-method", type=int, default=0)
    ap.add_argument("--rerank-mult", type=int, default=4)
    ap.add_argument("--d", type=int, default=128, choices=[128, 960])
    a = ap.parse_args()
    n = a.n or (1_000_000 if a.what == "search" else 200_000)
    X, Q, _ = synth.workload("mixture-1m-d128" if a.d == 128 else "mixture-1m-d960", n=n, nq=a.nq)
    Xd = torch.from_numpy(X).cuda()
    if a.what == "tiles":
        idx = H.Index(Xd, storage=H.BF16, seed=0, tiles=H.TILES_TCGEN05)
        info = idx.info()
        print("tiles ok", info["sizes"], f"tile_seconds={info['tile_seconds']:.4f}",
              f"uncertified={info['uncertified_rows']}")
        return
    Qd = torch.from_numpy(Q).cuda()
    idx = H.Index(Xd, storage=H.BF16, seed=0)
    for _ in range(3):
        ids, _, _ = idx.search(Qd, k=10, ef=a.ef, ef_upper=a.ef_upper, descend_all=a.descend_all, ef_l1=a.ef_l1,
                               exact_upper=a.exact_upper, exact_method=a.exact_method, rerank_mult=a.rerank_mult)
    torch.cuda.synchronize()
    print("search ok", idx.info()["sizes"], ids[0, :3].tolist())


if __name__ == "__main__":
    main()
