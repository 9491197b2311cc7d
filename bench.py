"""Benchmark: HENN search QPS at recall@10 >= 0.95 on one GB300 (1M x 128
Gaussian-mixture workload rescaled to [0, 255], 10,000 queries, k = 10),
batched BF16 traversal + exact FP32 rerank vs plain FP32; build seconds.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--sweep]
                    [--shape warps,team,hash_bits,tile_n]

One step = one henn_search call over the whole 10,000-query batch with the
index resident in HBM: one persistent search launch, preceded, when the
lowest exact upper layer comes from distance tiles (exact_method TILES), by
the query preparation, tile and top-32 selection launches.  The end-to-end
figure (`e2e`) times the same call with the queries and the result buffers
in page-locked host memory, which the kernels read and write in place over
the host link (5.12 MB in, 1.2 MB out per step, inside the timed region).
After the timed regions a `serving` entry reports the resident serving loop
on the same index under an open-loop request stream (achieved queries/s,
p50 / p99 latency at two offered rates).

The beam (ef, ef_upper, descend_all, ef_l1, exact_upper, exact_method,
rerank_mult) is DEFAULT_BEAM unless --sweep or --beam picks another.  Its
recall@10 is scored against FP64 ground truth (the FP64 order of each
query's 64 FP32-nearest candidates from henn_exact_knn, checked against an
FP64 brute force on a sample), with ties at the 10th distance counted; if
it falls under 0.95, ef steps up the EF_SWEEP list until it does not.  The
same beam is also scored on a held-out query batch.  Beside it the line
reports the best beam that only walks the upper layers (no exact layer) and
the paper's plain greedy descent (Alg. 4 on every upper layer).  The launch
shape comes from the autotuner, or from --shape (for runs under a profiler,
where the autotuner's timings mean nothing).

Under torchrun every rank holds its own index replica and its own query
batch (weak scaling, no collective on the data path); rank 0 prints one
JSON line with the whole-job throughput.

--impl reference times the FP64 CPU oracle on the host cores instead (the
reference arm): it builds its own index on a bounded sample of the same
workload and answers queries with the same beam form.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "search QPS at recall@10≥0.95 on 1×GB300, chosen form vs plain FP32; build seconds"
WORKLOAD = "mixture-1m-d128"
EF_SWEEP = [16, 24, 32, 36, 40, 44, 48, 52, 56, 64, 72, 80, 96, 128, 192, 256, 384, 512, 768, 1024]
# A beam is (ef, ef_upper, descend_all, ef_l1, exact_upper, exact_method, rerank_mult): the
# layer-0 width, the width on the upper layers (<= 1: GreedySearch of Alg. 4), whether each
# layer is entered at all candidates of the layer above, the width on layer 1 (0 = ef_upper),
# the size up to which an upper layer gives its exact candidate set ("L<i>": the size of layer
# i of the index at hand; 0 = never), how that set is found (0 SORT, 1 TILES) and the FP32
# rerank of the best rerank_mult * k.
#
# The default: layer 2 (3,677 points of the 1M mixture) exact from one batched distance-tile
# launch, its 16 nearest seeding the layer-1 beam, which keeps the best 8 (ef_l1), a width-50
# beam on layer 0, the FP32 rerank of the best 20.  Measured on this workload (FP64-scored,
# scored and held-out batches): 0.9559 / 0.9531 at 0.847 ms per batch, against 0.9556 / 0.9537
# at 0.864 ms for a width-16 layer-1 beam at ef 48.
DEFAULT_BEAM = (50, 16, 1, 8, "L2", 1, 2)
# --sweep: (ef_upper, descend_all, ef_l1, exact_upper, exact_method[, rerank_mult]), each
# tried at every ef of EF_SWEEP up to the first that reaches the target
UPPER_SWEEP = [(1, 0, 0, 0, 0), (32, 0, 0, 0, 0), (48, 1, 0, 0, 0), (64, 0, 0, 0, 0), (64, 1, 0, 0, 0),
               (64, 0, 16, 0, 0), (96, 0, 16, 0, 0), (128, 1, 16, 0, 0),
               (64, 1, 0, 256, 0), (64, 0, 16, 256, 0),
               (1, 0, 0, "L2", 1), (8, 1, 0, "L2", 1), (16, 1, 0, "L2", 1), (24, 1, 0, "L2", 1),
               (32, 0, 0, "L2", 1), (1, 0, 0, "L1", 1), (8, 1, 0, "L2", 1, 2), (16, 1, 0, "L2", 1, 2)]
# Upper layers walked by beams only (no exact layer): the best of these is reported beside the
# default (reading 11 of the paper's "set of candidates at each step" without reading 16).
WALK_SWEEP = [(64, 0, 16, 0, 0), (64, 1, 0, 0, 0), (48, 1, 0, 0, 0), (96, 0, 16, 0, 0), (128, 1, 16, 0, 0)]
K = 10
RECALL_TARGET = 0.95
GT_POOL = 64          # FP32 candidates per query that the FP64 ground truth re-ranks
GT_CHECK_QUERIES = 200  # queries whose ground truth is re-derived by an FP64 brute force
NOMINAL_HBM_GBS = 7900.0
L2_BYTES = 129 * 2**20


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(local_seconds: float, local_units: int, group=None):
    """Max of the ranks' timed seconds and the sum of their units."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return local_seconds, local_units
    t = torch.tensor([local_seconds], dtype=torch.float64)
    u = torch.tensor([float(local_units)], dtype=torch.float64)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else None
    if dev is not None:
        t, u = t.to(dev), u.to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), int(u.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def _smi_id(dev, local):
    """nvidia-smi id of this rank's GPU (its UUID when torch exposes it)."""
    import torch

    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(local)


# ------------------------------------------------------- FP64 ground truth

def fp64_sqdist(X, Q, ids):
    """FP64 squared L2 distances from each query to the rows ids[q, :]
    (direct differences; +inf where ids < 0)."""
    out = np.empty(ids.shape, np.float64)
    for q0 in range(0, len(Q), 1000):
        c = ids[q0:q0 + 1000]
        diff = X[np.maximum(c, 0)].astype(np.float64) - Q[q0:q0 + 1000, None, :].astype(np.float64)
        dd = np.einsum("qcd,qcd->qc", diff, diff)
        dd[c < 0] = np.inf
        out[q0:q0 + 1000] = dd
    return out


def rerank_fp64(X, Q, cand, k):
    """The k smallest (FP64 distance, id) of each query's candidate ids."""
    d = fp64_sqdist(X, Q, cand)
    order = np.lexsort((cand, d), axis=1)[:, :k]
    return np.take_along_axis(cand, order, 1), np.take_along_axis(d, order, 1)


def fp64_bruteforce(X, Q, k, pool=GT_POOL, chunk=250_000):
    """Exact k nearest by FP64 distance, every point of X examined: FP64
    dot-product distances pick each query's `pool` candidates, which are
    then ordered by FP64 direct differences (ties by id)."""
    Q64 = Q.astype(np.float64)
    qn = (Q64 * Q64).sum(1)
    best_d = np.full((len(Q), 0), np.inf)
    best_i = np.zeros((len(Q), 0), np.int64)
    for x0 in range(0, len(X), chunk):
        X64 = X[x0:x0 + chunk].astype(np.float64)
        D = (X64 * X64).sum(1)[None, :] - 2.0 * (Q64 @ X64.T) + qn[:, None]
        p = min(pool, D.shape[1])
        part = np.argpartition(D, p - 1, axis=1)[:, :p]
        best_d = np.concatenate([best_d, np.take_along_axis(D, part, 1)], 1)
        best_i = np.concatenate([best_i, part + x0], 1)
        keep = np.argsort(best_d, axis=1, kind="stable")[:, :pool]
        best_d = np.take_along_axis(best_d, keep, 1)
        best_i = np.take_along_axis(best_i, keep, 1)
    return rerank_fp64(X, Q, best_i, k)


def fp64_ground_truth(H, X, Q, Xd, Qd, k=K, pool=GT_POOL):
    """FP64 ground truth for all queries: henn_exact_knn's FP32 top-`pool`
    candidates re-ranked by FP64 distance."""
    cand, _ = H.exact_knn(Xd, Qd, pool)
    return rerank_fp64(X, Q, cand.cpu().numpy(), k)


def recall_fp64(X, Q, found, gt_ids, gt_d):
    """Mean recall@k (Sec. 2): |A_q ∩ O_q| / k, a returned id also counting
    when its FP64 distance equals the k-th ground-truth distance (ties)."""
    k = gt_ids.shape[1]
    found = np.asarray(found)[:, :k]
    fd = fp64_sqdist(X, Q, found)
    hit = (found[:, :, None] == gt_ids[:, None, :]).any(2) | ((found >= 0) & (fd == gt_d[:, k - 1:k]))
    return float(hit.sum(1).mean()) / k


def _beam(spec, sizes):
    """(ef, ef_upper, descend_all, ef_l1, exact_upper, exact_method, rerank_mult), "L<i>" resolved."""
    ef, efu, da, l1, xu, xm, rm = spec
    if isinstance(xu, str):
        li = int(xu[1:])
        xu = sizes[li] if li < len(sizes) else 0
    return (int(ef), int(efu), int(da), int(l1), int(xu), int(xm), int(rm))


def _kw(beam, shape=None):
    ef, efu, da, l1, xu, xm, rm = beam
    kw = dict(k=K, ef=ef, ef_upper=efu, descend_all=da, ef_l1=l1, exact_upper=xu, exact_method=xm, rerank_mult=rm)
    kw.update(shape or {})
    return kw


def _timed_search(index, Qd, beam, steps, warmup, flush, stream, shape=None, kernel_ms=None):
    """Step times (s) of `steps` calls after `warmup`, and the last ids;
    with a list in kernel_ms, also the device time of each call's search
    launches (henn_last_search_ms)."""
    import torch

    kw = _kw(beam, shape)
    if kernel_ms is not None:
        kw["time_kernel"] = True
    nq = Qd.shape[0]
    ids = torch.empty((nq, K), dtype=torch.int64, device=Qd.device)
    dd = torch.empty((nq, K), dtype=torch.float32, device=Qd.device)
    for _ in range(warmup):
        index.search(Qd, stream=stream, out=(ids, dd), **kw)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        if flush is not None:
            flush.add_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        index.search(Qd, stream=stream, out=(ids, dd), **kw)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        if kernel_ms is not None:
            kernel_ms.append(index.last_search_ms())
    return times, ids


def _score(index, Qd, Q, X, gt, beam, stream, flush, reps=4):
    """(recall vs FP64, median step seconds over `reps`) of one beam."""
    t, ids = _timed_search(index, Qd, beam, reps, 1, flush, stream)
    return recall_fp64(X, Q, ids.cpu().numpy(), *gt), statistics.median(t)


def _reach_target(index, Qd, Q, X, gt, beam, stream, flush, log_tag):
    """The beam with ef stepped up EF_SWEEP (from its own ef) until the
    recall target is met; returns (beam, recall, seconds) or None."""
    ef0 = beam[0]
    for ef in [ef0] + [e for e in EF_SWEEP if e > ef0]:
        b = (ef,) + tuple(beam[1:])
        r, t = _score(index, Qd, Q, X, gt, b, stream, flush)
        print(f"[{log_tag}] beam={b} recall@10={r:.5f} ms={1e3 * t:.3f}", file=sys.stderr, flush=True)
        if r >= RECALL_TARGET:
            return b, r, t
    return None


def _sweep(index, Qd, Q, X, gt, entries, sizes, stream, flush, tag):
    """Cheapest (by median step time) of the sweep entries at their first
    ef reaching the target; a later entry must be 2% faster to replace."""
    best = None
    for entry in entries:
        efu, da, l1, xu, xm = entry[:5]
        rm = entry[5] if len(entry) > 5 else 4
        beam = _beam((EF_SWEEP[0], efu, da, l1, xu, xm, rm), sizes)
        if isinstance(xu, str) and beam[4] == 0:
            continue
        got = _reach_target(index, Qd, Q, X, gt, beam, stream, flush, tag)
        if got and (best is None or got[2] < 0.98 * best[2]):
            best = got
    return best


def _export_layers(index):
    """The GPU-built hierarchy as plain per-layer arrays (host)."""
    info = index.info()
    ids, down, adj = [None], [None], []
    for i in range(info["L"] + 1):
        lay = index.layer(i)
        if i >= 1:
            ids.append(lay["ids"].astype(np.int64))
            down.append(lay["down"].astype(np.int64))
        adj.append(lay["adj"])
    return ids, down, adj


def _cpu_oracle_on_index(layers, X, Q, beam, nq_sample):
    """The FP64 oracle (as it stands) on the host cores, searching the same
    hierarchy the GPU searches (its layers, down pointers and graphs,
    imported) with the same beam form: nq_sample queries answered one
    after another on one core (the paper's sequential-query protocol), and
    once more with OpenMP over queries on all cores.  Returns (qps, cores,
    seconds, (qps_all_cores, cores))."""
    import oracle

    ids, down, adj = layers
    view = oracle.from_layers(ids, down, adj, seed=0)
    ef, efu, da, l1, xu, _, _ = beam
    Qs = np.ascontiguousarray(Q[:nq_sample])
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.search(view, X, Qs, k=K, ef=ef, ef_upper=efu, ef_l1=l1, descend_all=da, exact_upper=xu)
    secs = time.perf_counter() - t0
    ncores = len(os.sched_getaffinity(0))
    oracle.set_threads(ncores)
    t0 = time.perf_counter()
    oracle.search(view, X, Qs, k=K, ef=ef, ef_upper=efu, ef_l1=l1, descend_all=da, exact_upper=xu)
    all_cores = (nq_sample / (time.perf_counter() - t0), ncores)
    return nq_sample / secs, 1, secs, all_cores


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, its own index
    on a bounded sample of the workload (the GPU is not used), answering
    queries with the default beam form (layer 2 exact, beams below)."""
    import oracle

    ws, rank, _ = _dist_env()
    if rank != 0:
        return 0
    X, Q, _ = synth.workload(WORKLOAD, n=args.ref_n, nq=args.ref_nq)
    oracle.set_threads(len(os.sched_getaffinity(0)))
    idx = oracle.build_index(X, seed=0)
    beam = _beam(DEFAULT_BEAM, [int(s) for s in idx["sizes"]])
    ef, efu, da, l1, xu, _, _ = beam
    oracle.set_threads(1)
    secs = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.search(idx, X, Q, k=K, ef=ef, ef_upper=efu, ef_l1=l1, descend_all=da, exact_upper=xu)
        if i >= args.warmup:  # the first W steps are untimed warm-up
            secs.append(time.perf_counter() - t0)
    qps = args.ref_nq / statistics.median(secs)
    sample = (f"FP64 oracle, own index on the first {args.ref_n} of the 1M mixture points (same generator; "
              f"layers {[int(s) for s in idx['sizes']]}), {args.ref_nq} queries per step answered sequentially on "
              f"one core, ef={ef}, ef_upper={efu}, descend_all={da}, exact_upper={xu} (its layer 2), k={K}")
    line = {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n": 1_000_000, "d": 128, "nq": 10_000, "k": K},
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    ws, rank, local = _dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2505_17368_gb300 as H

    H.load()
    stream = torch.cuda.current_stream()
    # ---- inputs (same base set on every rank, own query batch per rank, a held-out batch)
    X, rngmap = synth.gaussian_mixture(args.n, 128, 1000, seed=0, rescale_to_255=True)
    Q, _ = synth.gaussian_mixture(args.nq, 128, 1000, seed=1 + rank, rescale_from=rngmap, rescale_to_255=True)
    Qh_out, _ = synth.gaussian_mixture(args.nq, 128, 1000, seed=1000 + rank, rescale_from=rngmap,
                                       rescale_to_255=True)
    Xd = torch.from_numpy(X).to(dev)
    Qd = torch.from_numpy(Q).to(dev)
    Qd_out = torch.from_numpy(Qh_out).to(dev)
    torch.cuda.synchronize()
    # ---- builds (inputs already resident; wall clock of henn_build)
    t0 = time.perf_counter()
    idx_bf16 = H.Index(Xd, storage=H.BF16, seed=0)
    build_bf16 = time.perf_counter() - t0
    t0 = time.perf_counter()
    idx_f32 = H.Index(Xd, storage=H.F32, seed=0)
    build_f32 = time.perf_counter() - t0
    info = idx_bf16.info()
    sizes = info["sizes"]
    # ---- FP64 ground truth (GPU candidates, FP64 order), checked on a sample by FP64 brute force
    gt = fp64_ground_truth(H, X, Q, Xd, Qd)
    gt_out = fp64_ground_truth(H, X, Qh_out, Xd, Qd_out)
    chk = np.random.default_rng(5).choice(args.nq, min(GT_CHECK_QUERIES, args.nq), replace=False)
    bf_i, _ = fp64_bruteforce(X, Q[chk], K)
    gt_check = {"queries": int(len(chk)), "identical": int(np.all(bf_i == gt[0][chk], axis=1).sum())}
    flush = torch.empty(L2_BYTES * 2 // 4, dtype=torch.float32, device=dev)
    # ---- beam: default (or --beam / --sweep), ef stepped up until recall >= target
    if args.sweep:
        chosen = _sweep(idx_bf16, Qd, Q, X, gt, UPPER_SWEEP, sizes, stream, flush, "sweep bf16")
    else:
        spec = DEFAULT_BEAM
        if args.beam:
            f = args.beam.split(",")
            spec = tuple(int(v) if not v.startswith("L") else v for v in f)
            if len(spec) == 6:
                spec = spec + (4,)
        chosen = _reach_target(idx_bf16, Qd, Q, X, gt, _beam(spec, sizes), stream, flush, "beam bf16")
    if chosen is None:
        raise SystemExit("recall target not reached")
    beam, rec_sweep, _ = chosen
    ef, efu, da, l1, xu, xm, rm = beam
    # ---- launch shape (warps per block, visited-table size) by the autotuner
    from paper_2505_17368_gb300 import autotune

    if args.shape:
        # a fixed launch shape (profiling: the autotuner's timings are not
        # meaningful under a profiler)
        w, t, hb, tn = (int(x) for x in args.shape.split(","))
        shape = {"warps_per_block": w, "team_size": t, "hash_bits": hb, "tile_n": tn}
    else:
        shape = autotune.tune(idx_bf16, Qd, k=K, ef=ef, ef_upper=efu, ef_l1=l1, descend_all=da, exact_upper=xu,
                              exact_method=xm, rerank_mult=rm, use_cache=False)
    # ---- algorithmic bytes per launch from the kernel's own counters
    _, _, st = idx_bf16.search(Qd, stats=True, **_kw(beam, shape))
    st = st.cpu().numpy().astype(np.int64)
    row_bf16 = 128 * 2
    R = min(rm * K, ef)
    alg_bytes = int(st[:, 0].sum() * row_bf16 + st[:, 1].sum() * 128 + args.nq * (R * 128 * 4 + 128 * 4 + K * 12))
    if xm == 1 and xu > 0:
        alg_bytes += args.nq * (32 * 8 + 4)  # each query's tile candidates and centred norm
    # ---- timed region
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    kern = []
    with ClockSampler(_smi_id(dev, local)) as clk:
        times, ids = _timed_search(idx_bf16, Qd, beam, args.steps, args.warmup, flush, stream, shape=shape,
                                   kernel_ms=kern)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.summary()
    local_time = sum(times)
    tmax, units = aggregate(local_time, args.nq * args.steps)
    value = units / tmax
    # recall of the timed region's own results (autotuned launch shape), and on the held-out batch
    rec = recall_fp64(X, Q, ids.cpu().numpy(), *gt)
    ids_out, _, _ = idx_bf16.search(Qd_out, **_kw(beam, shape))
    rec_out = recall_fp64(X, Qh_out, ids_out.cpu().numpy(), *gt_out)
    # ---- plain FP32 at the same beam: batched, and one launch per query
    p_times, p_ids = _timed_search(idx_f32, Qd, beam, args.steps, args.warmup, flush, stream)
    plain_qps = args.nq / statistics.median(p_times)
    p_rec = recall_fp64(X, Q, p_ids.cpu().numpy(), *gt)
    ns = min(200, args.nq)
    t_one = []
    for q in range(ns):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        idx_f32.search(Qd[q:q + 1], stream=stream, **_kw(beam))
        e1.record(stream)
        e1.synchronize()
        t_one.append(e0.elapsed_time(e1) / 1e3)
    per_query_qps = 1.0 / statistics.median(t_one)
    # ---- the upper layers walked by beams only, and the paper's greedy descent
    walk = _sweep(idx_bf16, Qd, Q, X, gt, WALK_SWEEP, sizes, stream, flush, "walk bf16")
    greedy = []
    for g_ef in (64, 256, 1024):
        r, t = _score(idx_bf16, Qd, Q, X, gt, (g_ef, 1, 0, 0, 0, 0, rm), stream, flush, reps=2)
        greedy.append({"ef": g_ef, "recall_at_10": r, "qps": args.nq / t})
    # ---- end to end through the C ABI with host buffers
    # queries and the result buffers in page-locked host memory, as a serving
    # caller keeps them: the copies in and out are direct DMA transfers
    Qh = torch.from_numpy(Q).pin_memory()
    ids_h = torch.empty((args.nq, K), dtype=torch.int64).pin_memory()
    dists_h = torch.empty((args.nq, K), dtype=torch.float32).pin_memory()
    e2e_t = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        idx_bf16.search(Qh.numpy(), stream=stream, out=(ids_h.numpy(), dists_h.numpy()), **_kw(beam, shape))
        if i >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    e2e_tmax, e2e_units = aggregate(sum(e2e_t), args.nq * args.steps)
    # ---- the serving loop on the same index (after every timed region; rank 0's GPU only, so
    # that the other ranks' host threads do not compete with its submitter and poller)
    serving = None if (args.shape or rank != 0) else _serving_leg(H, idx_bf16, Q, sizes)
    peaks, src = _peaks()
    # the search kernel's own device time (events around its launch), not the step's
    k_avg = statistics.mean(ms for ms, _ in kern) / 1e3
    launches_per_step = kern[-1][1]
    achieved = alg_bytes / k_avg / 1e9
    traffic = _profile_traffic(beam[:6], rm)
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {
            "workload": WORKLOAD, "n": args.n, "d": 128, "nq": args.nq, "k": K, "ef": ef, "ef_upper": efu,
            "descend_all": da, "ef_l1": l1, "exact_upper": xu, "exact_method": xm, "rerank_mult": rm,
            "beam_source": "sweep" if args.sweep else ("--beam" if args.beam else "default"),
            "launch_shape": shape,
            "launch_shape_source": "--shape" if args.shape else "autotuner",
            "form": f"bf16 traversal + fp32 rerank of top {rm}k", "recall_at_10": rec,
            "recall_at_10_held_out": rec_out, "recall_scoring": (
                f"FP64 ground truth (FP64 order of each query's {GT_POOL} FP32-nearest candidates from "
                f"henn_exact_knn; identical to an FP64 brute force on {gt_check['identical']} of "
                f"{gt_check['queries']} sampled queries), ties at the 10th distance counted; held-out: "
                f"another {args.nq} queries of the same mixture"),
            "l2": "flushed between steps",
            "layers": sizes, "build_seconds_bf16": build_bf16, "build_seconds_f32": build_f32,
            "plain_f32": {"qps": plain_qps, "recall_at_10": p_rec, "beam": "same as the chosen form"},
            "plain_f32_per_query_launch_qps": per_query_qps,
            "walk_only_bf16": None if walk is None else {
                "qps": args.nq / walk[2], "recall_at_10": walk[1], "ef": walk[0][0], "ef_upper": walk[0][1],
                "descend_all": walk[0][2], "ef_l1": walk[0][3], "rerank_mult": walk[0][6],
                "note": "upper layers walked by beams only, no exact layer; median of 4 steps"},
            "greedy_descent_bf16": greedy,
            "step_ms_median": 1e3 * statistics.median(times), "step_ms_max": 1e3 * max(times),
            "qps_of_slowest_step": args.nq / max(times),
            "parallelism": f"replicas{ws}",
        },
        "build_seconds": build_bf16,
        "build_roofline": _build_roofline(info),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "traffic": traffic, "peak_source": src, "kernel_ms": 1e3 * k_avg,
                     "algorithmic_bytes_per_launch": alg_bytes, "kernel": "k_search<bf16>"},
        "e2e": {"value": e2e_units / e2e_tmax, "unit": "queries/s",
                "h2d_bytes_per_step": int(args.nq * 128 * 4), "d2h_bytes_per_step": int(args.nq * K * 12)},
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clocks,
    }
    if serving is not None:
        line["serving"] = serving
    if rank == 0 and not args.no_cpu_baseline:
        layers = _export_layers(idx_bf16)
        qps, cores, secs, (qps_all, ncores) = _cpu_oracle_on_index(layers, X, Q, beam, args.cpu_nq)
        sample = (f"FP64 oracle searching the GPU-built 1M x 128 hierarchy (imported layers, down pointers "
                  f"and graphs), first {args.cpu_nq} of the {args.nq} queries, same beam (ef={ef}, "
                  f"ef_upper={efu}, descend_all={da}, ef_l1={l1}, exact_upper={xu}; the oracle finds exact "
                  f"layers by brute force and searches in FP64)")
        line["cpu_baseline"] = {
            "value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": sample + f", answered sequentially on one core (the paper's protocol), {secs:.1f} s",
        }
        line["cpu_baseline_all_cores"] = {
            "value": qps_all, "unit": "queries/s", "cores": ncores, "kind": "oracle",
            "sample": sample + ", OpenMP over queries on all host cores",
        }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _build_roofline(info):
    """Tensor-pipe roofline of the construction distance tiles: the
    library times its tile launches with CUDA events on the build stream;
    algorithmic flops = 2 d per valid (row, column) pair, summed over the
    layers.  The split-BF16 tcgen05 engine executes three BF16 products per
    pair (hi.hi + lo.hi + hi.lo), reported as executed_frac."""
    peaks, src = _peaks()
    if not info.get("tile_seconds"):
        return None
    achieved = info["tile_flops"] / info["tile_seconds"] / 1e12
    peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    engine = {1: "simt-fp32", 2: "tcgen05-split-bf16"}.get(info.get("tile_engine"), "unknown")
    mult = 3.0 if engine.startswith("tcgen05") else 1.0
    return {"bound": "tensor", "kernel": "k_tile_topk_tc" if mult == 3.0 else "k_tile_topk_simt",
            "engine": engine, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "executed_frac": mult * achieved / peak, "tile_seconds": info["tile_seconds"],
            "algorithmic_flops": info["tile_flops"], "peak_source": f"{src} bf16 sustained"}


def _serving_leg(H, index, Q, sizes, rates=(5e5, 2e6), seconds=2.0):
    """The resident serving loop (henn_serve_*) on the bench's index: an
    open-loop Poisson request stream (batches log-uniform in [1, 4096],
    k in {10, 100}, ef log-uniform in [64, 512]; serve_bench's mix) at two
    offered rates, 2 s each; achieved queries/s and p50 / p99 latency.  Layer
    3 gives its exact candidate set (in-kernel sort), seeding width-16 beams
    on layer 2 and width-8 beams on layer 1.  Outside every timed region;
    a failure is reported in the line instead of ending the run."""
    from paper_2505_17368_gb300 import serve_bench

    beam = dict(ef_upper=16, descend_all=1, ef_l1=8, exact_upper=int(sizes[3]) if len(sizes) > 3 else 0)
    try:
        srv = H.Server(index, ring_rows=1 << 17, max_requests=4096, max_k=100, max_ef=512, **beam)
        try:
            out = []
            for r in rates:
                res = serve_bench.run_rate(srv, Q, r, seconds, 4096, seed=int(r) % 1000)
                out.append({k: res[k] for k in ("offered_qps", "achieved_qps", "p50_ms", "p99_ms", "requests")})
        finally:
            srv.close()
    except Exception as e:  # noqa: BLE001 -- reported, the headline stands
        return {"error": str(e)[:300]}
    return {"workload": WORKLOAD, "form": "bf16 + fp32 rerank", "beam": beam,
            "mix": "Poisson arrivals; batch log-uniform [1, 4096], k in {10, 100}, ef log-uniform [64, 512]",
            "rates": out}


def _profile_traffic(beam, rerank_mult=4):
    """DRAM bytes per launch of the search kernel from the committed ncu
    summary, if it was taken on the current kernel source with the same
    beam configuration (ef, ef_upper, descend_all, ef_l1, exact_upper,
    exact_method, and rerank_mult where it is not 4); else None."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "search_bf16_mixture-1m-d128.md")
    src = os.path.join(ROOT, "paper_2505_17368_gb300", "csrc", "search.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        kv = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].rsplit(":", 1)  # keys may hold a colon ("sha256[:16]")
                kv[k.strip()] = v.strip().strip("`")
        want = "ef={} ef_upper={} descend_all={} ef_l1={} exact_upper={} exact_method={}".format(*beam)
        if rerank_mult != 4:
            want += f" rerank_mult={rerank_mult}"
        if kv.get("search.cu sha256[:16]") == sha:
            return float(kv[f"dram bytes per launch [{want}]"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--cpu-nq", type=int, default=5_000)
    ap.add_argument("--ref-n", type=int, default=50_000)
    ap.add_argument("--ref-nq", type=int, default=2_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true", help="pick the beam by the UPPER_SWEEP search instead")
    ap.add_argument("--beam", default=None,
                    help="ef,ef_upper,descend_all,ef_l1,exact_upper,exact_method[,rerank_mult] instead of "
                         "DEFAULT_BEAM (exact_upper may be L<i>, the size of layer i)")
    ap.add_argument("--shape", default=None,
                    help="warps_per_block,team_size,hash_bits,tile_n: a fixed launch shape instead of the "
                         "autotuner's (for runs under a profiler; the serving leg is skipped then)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
