"""FP64 CPU oracle for HENN (arXiv 2505.17368) -- TEST INFRASTRUCTURE ONLY.

The oracle is the slow, literal statement of what the GPU path computes
(henn_oracle.c).  Only the test-suite, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import it; the product package never does.
This module compiles the C source with gcc and wraps it with ctypes/numpy.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "henn_oracle.c")
_HDR = os.path.join(_HERE, "henn_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libhenn_oracle.so")
_lock = threading.Lock()
_lib = None

L2, ANGULAR = 0, 1
GRAPH_NSW, GRAPH_KNN = 0, 1
SAMPLER_SAMPLING, SAMPLER_HALVING = 0, 1  # Alg. 2 (sampling + verification) or Alg. 3 V2 (halving)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C11, FP64, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    fresh = os.path.exists(_OUT) and os.path.getmtime(_OUT) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)
    )
    if force or not fresh:
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
             _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _OUT)
    return _OUT


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.ho_set_threads.restype = None
            L.ho_set_threads.argtypes = [C.c_int32]
            L.ho_mix64.restype = C.c_uint64
            L.ho_mix64.argtypes = [C.c_uint64]
            L.ho_derive.restype = C.c_uint64
            L.ho_derive.argtypes = [C.c_uint64, C.c_uint64]
            L.ho_bounded.restype = C.c_uint64
            L.ho_bounded.argtypes = [C.c_uint64, C.c_uint64]
            L.ho_order_rank.restype = C.c_int64
            L.ho_order_rank.argtypes = [C.c_uint64, C.c_int32, C.c_int64, C.c_int64]
            L.ho_ring_window.restype = C.c_int64
            L.ho_ring_window.argtypes = [C.c_double, C.c_int32, C.c_int64, C.c_int32]
            L.ho_dist.restype = C.c_double
            L.ho_dist.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32, C.c_int32]
            L.ho_sample_positions.restype = C.c_int64
            L.ho_sample_positions.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_int64, C.c_int64,
                                              C.POINTER(C.c_int64)]
            L.ho_verify.restype = C.c_int32
            L.ho_verify.argtypes = [C.POINTER(C.c_float), C.c_int32, C.c_int32, C.POINTER(C.c_int64),
                                    C.c_int64, C.POINTER(C.c_int64), C.c_int64, C.c_uint64, C.c_int32,
                                    C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_uint8)]
            L.ho_build_layers_from.restype = C.c_int32
            L.ho_build_layers_from.argtypes = [C.POINTER(C.c_float), C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                               C.c_double, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, C.c_int32,
                                               C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64),
                                               C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
            L.ho_build_layers_halving.restype = C.c_int32
            L.ho_build_layers_halving.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_uint64,
                                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.ho_halving_positions.restype = C.c_int64
            L.ho_halving_positions.argtypes = [C.c_uint64, C.c_int32, C.c_int64, C.c_int32, C.POINTER(C.c_int64)]
            L.ho_build_layers.restype = C.c_int32
            L.ho_build_layers.argtypes = [C.POINTER(C.c_float), C.c_int64, C.c_int32, C.c_int32,
                                          C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                          C.c_uint64, C.c_int32, C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int32)]
            L.ho_forward_lists.restype = None
            L.ho_forward_lists.argtypes = [C.POINTER(C.c_float), C.c_int32, C.c_int32,
                                           C.POINTER(C.c_int64), C.c_int64, C.c_uint64, C.c_int32,
                                           C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                           C.POINTER(C.c_double)]
            L.ho_forward_row.restype = None
            L.ho_forward_row.argtypes = [C.POINTER(C.c_float), C.c_int32, C.c_int32,
                                         C.POINTER(C.c_int64), C.c_int64, C.c_uint64, C.c_int32,
                                         C.c_int32, C.c_int32, C.c_int64, C.POINTER(C.c_int32),
                                         C.POINTER(C.c_double)]
            L.ho_edge_rule.restype = None
            L.ho_edge_rule.argtypes = [C.POINTER(C.c_int32), C.POINTER(C.c_double), C.c_int64,
                                       C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
            L.ho_search.restype = None
            L.ho_search.argtypes = [C.POINTER(C.c_float), C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_float), C.c_int64,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int32,
                                    C.c_int64, C.c_uint64,
                                    C.POINTER(C.c_uint64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_int64)]
            L.ho_greedy_layer.restype = C.c_int64
            L.ho_greedy_layer.argtypes = [C.POINTER(C.c_float), C.c_int32, C.c_int32,
                                          C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_int32,
                                          C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int64)]
            L.ho_bruteforce.restype = None
            L.ho_bruteforce.argtypes = [C.POINTER(C.c_float), C.c_int64, C.c_int32, C.c_int32,
                                        C.POINTER(C.c_float), C.c_int64, C.c_int32,
                                        C.POINTER(C.c_int64), C.POINTER(C.c_double)]
            L.ho_bf16_bits.restype = C.c_uint16
            L.ho_bf16_bits.argtypes = [C.c_float]
            L.ho_e4m3_bits.restype = C.c_uint8
            L.ho_e4m3_bits.argtypes = [C.c_float]
            L.ho_e4m3_value.restype = C.c_double
            L.ho_e4m3_value.argtypes = [C.c_uint8]
        return _lib


def _f32(X):
    return np.ascontiguousarray(X, dtype=np.float32)


def set_threads(n: int) -> None:
    """OpenMP threads for the oracle's row / query loops."""
    lib().ho_set_threads(int(n))


# ----------------------------------------------------------------- RNG

def mix64(z: int) -> int:
    return lib().ho_mix64(z & 0xFFFFFFFFFFFFFFFF)


def derive(h: int, w: int) -> int:
    return lib().ho_derive(h & 0xFFFFFFFFFFFFFFFF, w & 0xFFFFFFFFFFFFFFFF)


def bounded(u: int, s: int) -> int:
    return lib().ho_bounded(u & 0xFFFFFFFFFFFFFFFF, s)


def order_ranks(seed: int, layer: int, s: int) -> np.ndarray:
    f = lib().ho_order_rank
    return np.array([f(seed, layer, s, x) for x in range(s)], dtype=np.int64)


def ring_window(c0: float, d: int, s: int, m: int) -> int:
    return lib().ho_ring_window(c0, d, s, m)


def dist(a, b, metric=L2) -> float:
    a, b = _f32(a), _f32(b)
    return lib().ho_dist(_p(a, C.c_float), _p(b, C.c_float), a.shape[-1], metric)


# ------------------------------------------------------------ layers

def sample_positions(seed: int, layer: int, attempt: int, s: int, t: int) -> np.ndarray:
    out = np.empty(max(t, 1), dtype=np.int64)
    cnt = lib().ho_sample_positions(seed, layer, attempt, s, t, _p(out, C.c_int64))
    return out[:cnt].copy()


def verify(X, prev, net_pos, seed, layer, attempt, r, w, metric=L2, exhaustive=False):
    X = _f32(X)
    prev = np.ascontiguousarray(prev, dtype=np.int64)
    net_pos = np.ascontiguousarray(net_pos, dtype=np.int64)
    ring_ok = np.zeros(max(r, 1), dtype=np.uint8)
    ok = lib().ho_verify(_p(X, C.c_float), X.shape[1], metric, _p(prev, C.c_int64), len(prev),
                         _p(net_pos, C.c_int64), len(net_pos), seed, layer, attempt, r, w,
                         int(exhaustive), _p(ring_ok, C.c_uint8))
    return bool(ok), ring_ok[:r].astype(bool)


def halving_positions(s, m, seed, layer):
    """Alg. 3 (BuildEpsNetDiscV2) on positions 0..s-1: the survivors."""
    out = np.zeros(max(s, 1), dtype=np.int64)
    c = lib().ho_halving_positions(seed, layer, s, m, _p(out, C.c_int64))
    return out[:c].copy()


def build_layers(X, m=4, max_layers=0, c0=1.0, r=100, max_attempts=64, seed=0, metric=L2,
                 exhaustive=False, sampler=SAMPLER_SAMPLING):
    """Layer membership (Alg. 1 + Alg. 2, or Alg. 3 halving).  Returns dict
    or raises RuntimeError."""
    X = _f32(X)
    n, d = X.shape
    sizes = np.zeros(64, dtype=np.int64)
    ids = np.zeros(max(n, 1), dtype=np.int64)
    down = np.zeros(max(n, 1), dtype=np.int64)
    attempts = np.zeros(64, dtype=np.int32)
    if sampler == SAMPLER_HALVING:
        L = lib().ho_build_layers_halving(n, m, max_layers, seed, _p(sizes, C.c_int64), _p(ids, C.c_int64),
                                          _p(down, C.c_int64))
    else:
        L = lib().ho_build_layers(_p(X, C.c_float), n, d, metric, m, max_layers, c0, r, max_attempts,
                                  seed, int(exhaustive), _p(sizes, C.c_int64), _p(ids, C.c_int64),
                                  _p(down, C.c_int64), _p(attempts, C.c_int32))
    if L < 0:
        raise RuntimeError("no epsilon-net found within max_attempts")
    layer_ids, layer_down = [np.arange(n, dtype=np.int64)], [None]
    off = 0
    for i in range(1, L + 1):
        s = int(sizes[i])
        layer_ids.append(ids[off:off + s].copy())
        layer_down.append(down[off:off + s].copy())
        off += s
    return dict(L=L, sizes=sizes[:L + 1].copy(), ids=layer_ids, down=layer_down,
                attempts=attempts[:L + 1].copy())


def forward_lists(X, ids, seed, layer, M=16, graph=GRAPH_NSW, metric=L2):
    X = _f32(X)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    s = len(ids)
    fwd = np.empty((max(s, 1), M), dtype=np.int32)
    fwd_d = np.empty((max(s, 1), M), dtype=np.float64)
    lib().ho_forward_lists(_p(X, C.c_float), X.shape[1], metric, _p(ids, C.c_int64), s, seed, layer,
                           M, graph, _p(fwd, C.c_int32), _p(fwd_d, C.c_double))
    return fwd[:s], fwd_d[:s]


def forward_row(X, ids, seed, layer, p, M=16, graph=GRAPH_NSW, metric=L2):
    X = _f32(X)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    fwd = np.empty(M, dtype=np.int32)
    fwd_d = np.empty(M, dtype=np.float64)
    lib().ho_forward_row(_p(X, C.c_float), X.shape[1], metric, _p(ids, C.c_int64), len(ids), seed, layer, M,
                         graph, int(p), _p(fwd, C.c_int32), _p(fwd_d, C.c_double))
    return fwd, fwd_d


def edge_rule(fwd, fwd_d, Mmax=32, graph=GRAPH_NSW):
    fwd = np.ascontiguousarray(fwd, dtype=np.int32)
    fwd_d = np.ascontiguousarray(fwd_d, dtype=np.float64)
    s, M = fwd.shape
    adj = np.empty((max(s, 1), Mmax), dtype=np.int32)
    lib().ho_edge_rule(_p(fwd, C.c_int32), _p(fwd_d, C.c_double), s, M, Mmax, graph,
                       _p(adj, C.c_int32))
    return adj[:s]


def build_index(X, m=4, max_layers=0, c0=1.0, r=100, max_attempts=64, seed=0, M=16, Mmax=32,
                graph=GRAPH_NSW, metric=L2, exhaustive=False, sampler=SAMPLER_SAMPLING):
    """Full HENN (Alg. 1): layers, per-layer forward lists and adjacency."""
    idx = build_layers(X, m, max_layers, c0, r, max_attempts, seed, metric, exhaustive, sampler)
    idx["fwd"], idx["fwd_d"], idx["adj"] = [], [], []
    for i, ids in enumerate(idx["ids"]):
        f, fd = forward_lists(X, ids, seed, i, M, graph, metric)
        idx["fwd"].append(f)
        idx["fwd_d"].append(fd)
        idx["adj"].append(edge_rule(f, fd, Mmax, graph))
    idx.update(M=M, Mmax=Mmax, seed=seed, metric=metric, graph=graph)
    return idx


def from_layers(ids, down, adj, metric=L2, seed=0, M=16, Mmax=32, graph=GRAPH_NSW):
    """An index in this module's form from plain per-layer arrays (layer 0
    first): ids[i] the sorted global ids of layer i (ids[0] may be None for
    0..n-1), down[i] the positions of layer i in layer i-1 (down[0]
    ignored), adj[i] the |L_i| x Mmax layer-local adjacency rows.  Lets the
    oracle's search (Alg. 4 + beam) run on a hierarchy built elsewhere, such
    as the GPU's, so the two searches see the same layers and graphs."""
    L = len(adj) - 1
    n = len(adj[0])
    lid = [np.arange(n, dtype=np.int64)] + [np.asarray(ids[i], dtype=np.int64) for i in range(1, L + 1)]
    ldn = [None] + [np.asarray(down[i], dtype=np.int64) for i in range(1, L + 1)]
    ladj = [np.ascontiguousarray(a, dtype=np.int32) for a in adj]
    return dict(L=L, sizes=np.array([len(a) for a in lid], dtype=np.int64), ids=lid, down=ldn, adj=ladj,
                attempts=np.zeros(L + 1, np.int32), M=M, Mmax=Mmax, seed=seed, metric=metric, graph=graph)


TAG_INSERT = 0x494E5352  # "INSR": layer promotion coin of an inserted point (App. C, Insert)


def insert_layers(seed, p, m, L):
    """Layers an inserted point joins (App. C, Insert): layer 0, then layer i
    while the point is in layer i-1 and its coin bounded(derive(derive(
    derive(seed, INSR), p), i), 2^m) is 0 (each layer keeps about a 2^-m
    fraction of the one below, the rate of the built layers); at most L."""
    out = [0]
    for i in range(1, L + 1):
        if bounded(derive(derive(derive(seed, TAG_INSERT), p), i), 1 << m) != 0:
            break
        out.append(i)
    return out


def _dist64(X, p, members, metric):
    x = X[p].astype(np.float64)
    Y = X[members].astype(np.float64)
    if metric == ANGULAR:
        nx = math.sqrt(float(x @ x))
        ny = np.sqrt((Y * Y).sum(1))
        return 1.0 - (Y @ x) / (np.maximum(ny, 1e-300) * max(nx, 1e-300))
    return ((Y - x) ** 2).sum(1)


def insert(idx, X, new_ids, m=4):
    """Dynamic Insert (App. C) of the points `new_ids` (ascending, every id
    larger than the indexed ones; X holds all points), one after another.
    For each layer the point joins: it is appended to the layer (ids stay
    ascending), its down pointer is its position in the layer below, its
    forward list is the M nearest current members by (distance, position)
    (it is the last point in the layer's insertion order, so every member
    is earlier), and the layer's adjacency is the edge rule over the updated
    forward lists.  NSW graphs only.  Modifies and returns idx."""
    if idx["graph"] != GRAPH_NSW:
        raise ValueError("insert supports NSW graphs")
    X = _f32(X)
    M, Mmax, metric, L = idx["M"], idx["Mmax"], idx["metric"], idx["L"]
    for p in [int(v) for v in new_ids]:
        for i in insert_layers(idx["seed"], p, m, L):
            members = idx["ids"][i]
            s = len(members)
            d = _dist64(X, p, members, metric)
            order = np.lexsort((np.arange(s), d))[:M]
            row = np.full(M, -1, np.int32)
            row_d = np.full(M, np.inf)
            row[:len(order)] = order
            row_d[:len(order)] = d[order]
            idx["ids"][i] = np.append(members, p).astype(np.int64)
            if i >= 1:
                idx["down"][i] = np.append(idx["down"][i], len(idx["ids"][i - 1]) - 1).astype(np.int64)
            idx["fwd"][i] = np.vstack([idx["fwd"][i], row[None, :]])
            idx["fwd_d"][i] = np.vstack([idx["fwd_d"][i], row_d[None, :]])
            idx["adj"][i] = edge_rule(idx["fwd"][i], idx["fwd_d"][i], Mmax, idx["graph"])
        idx["sizes"] = np.array([len(a) for a in idx["ids"]], dtype=np.int64)
    return idx


def build_layers_from(X, prev_ids, first_layer, m=4, max_layers=0, c0=1.0, r=100, max_attempts=64, seed=0,
                      metric=L2):
    """Layers first_layer, first_layer + 1, ... (Alg. 1 + Alg. 2) built on
    top of a layer whose points are prev_ids (ascending global ids).
    Returns (ids per new layer, down per new layer -- positions in
    prev_ids for the first --, attempts per new layer); raises if no
    epsilon-net is found."""
    X = _f32(X)
    prev = np.ascontiguousarray(prev_ids, dtype=np.int64)
    s0 = len(prev)
    sizes = np.zeros(64, dtype=np.int64)
    ids = np.zeros(max(s0, 1), dtype=np.int64)
    down = np.zeros(max(s0, 1), dtype=np.int64)
    attempts = np.zeros(64, dtype=np.int32)
    top = lib().ho_build_layers_from(_p(X, C.c_float), X.shape[1], metric, m, max_layers, c0, r, max_attempts, seed,
                                     0, first_layer, _p(prev, C.c_int64), s0, _p(sizes, C.c_int64),
                                     _p(ids, C.c_int64), _p(down, C.c_int64), _p(attempts, C.c_int32))
    if top < 0:
        raise RuntimeError("no epsilon-net found within max_attempts")
    out_ids, out_down, out_att, off = [], [], [], 0
    for layer in range(first_layer, top + 1):
        c = int(sizes[layer])
        out_ids.append(ids[off:off + c].copy())
        out_down.append(down[off:off + c].copy())
        out_att.append(int(attempts[layer]))
        off += c
    return out_ids, out_down, out_att


def delete(idx, X, dead, m=4, max_layers=0, c0=1.0, r=100, max_attempts=64, share=0.5):
    """Delete of App. C on top of tombstones: `dead` (a boolean mask over
    global ids) holds every deleted point; deleted points stay in the
    layers as walk-only nodes and never come back (search(deleted=)).  The
    lowest upper layer i whose live points fall below `share` times the
    size a fresh sample of the live points of layer i - 1 would draw,
    ceil(live(L_{i-1}) / 2^m), is resampled from those live points (Alg. 2
    with the build's seed and layer numbers) and the hierarchy is rebuilt
    from it up to the root: membership, down pointers (positions in layer
    i - 1, whose arrays keep their dead entries) and graphs.  Layer 0 keeps
    every point.  Modifies idx; returns the first rebuilt layer or None."""
    X = _f32(X)
    dead = np.asarray(dead, dtype=bool)
    seed, M, Mmax, graph, metric = idx["seed"], idx["M"], idx["Mmax"], idx["graph"], idx["metric"]
    for i in range(1, idx["L"] + 1):
        below = idx["ids"][i - 1]
        livep = np.nonzero(~dead[below])[0]
        need = -(-len(livep) // (1 << m))
        if (~dead[idx["ids"][i]]).sum() >= share * need:
            continue
        new_ids, new_down, new_att = build_layers_from(X, below[livep], i, m, max_layers, c0, r, max_attempts, seed,
                                                       metric)
        idx["ids"] = idx["ids"][:i] + new_ids
        idx["down"] = idx["down"][:i] + ([livep[new_down[0]]] + new_down[1:] if new_ids else [])
        idx["attempts"] = np.concatenate([np.asarray(idx["attempts"][:i]), np.asarray(new_att, np.int32)])
        idx["fwd"], idx["fwd_d"], idx["adj"] = idx["fwd"][:i], idx["fwd_d"][:i], idx["adj"][:i]
        for j, lids in enumerate(new_ids):
            f, fd = forward_lists(X, lids, seed, i + j, M, graph, metric)
            idx["fwd"].append(f)
            idx["fwd_d"].append(fd)
            idx["adj"].append(edge_rule(f, fd, Mmax, graph))
        idx["L"] = i - 1 + len(new_ids)
        idx["sizes"] = np.array([len(a) for a in idx["ids"]], dtype=np.int64)
        return i
    return None


def search(idx, X, Q, k=10, ef=64, keys=None, out_stride=None, seed=None, ef_upper=1, ef_l1=0,
           descend_all=0, exact_upper=0, deleted=None):
    """Alg. 4 descent + layer-0 beam.  Returns (ids int64, dists f64, stats).
    deleted: optional boolean mask over global ids (Delete of App. C as
    tombstones): deleted points still carry the walk but the result is the
    first k live entries of the final candidate list."""
    if deleted is not None:
        kq = np.broadcast_to(np.asarray(k, dtype=np.int32), (Q.shape[0],)).copy()
        efq = np.broadcast_to(np.asarray(ef, dtype=np.int32), (Q.shape[0],)).copy()
        full = np.maximum(kq, efq)
        wi, wd, st = search(idx, X, Q, k=full, ef=efq, keys=keys, out_stride=int(full.max()), seed=seed,
                            ef_upper=ef_upper, ef_l1=ef_l1, descend_all=descend_all, exact_upper=exact_upper)
        stride = int(out_stride or max(int(kq.max()), 1))
        oi = np.full((len(Q), stride), -1, np.int64)
        od = np.full((len(Q), stride), np.inf)
        for q in range(len(Q)):
            live = [(i, v) for i, v in zip(wi[q], wd[q]) if i >= 0 and not deleted[i]][:kq[q]]
            for j, (i, v) in enumerate(live):
                oi[q, j], od[q, j] = i, v
        return oi, od, st
    X, Q = _f32(X), _f32(Q)
    n, d = X.shape
    nq = Q.shape[0]
    kq = np.broadcast_to(np.asarray(k, dtype=np.int32), (nq,)).copy()
    efq = np.broadcast_to(np.asarray(ef, dtype=np.int32), (nq,)).copy()
    stride = int(out_stride or max(int(kq.max()) if nq else 1, 1))
    L = idx["L"]
    sizes = np.ascontiguousarray(idx["sizes"], dtype=np.int64)
    ids = np.ascontiguousarray(np.concatenate([np.zeros(0, np.int64)] + list(idx["ids"][1:])), dtype=np.int64)
    down = np.ascontiguousarray(np.concatenate([np.zeros(0, np.int64)] + list(idx["down"][1:])), dtype=np.int64)
    Mmax = idx["Mmax"]
    adj = np.ascontiguousarray(np.concatenate([a.reshape(-1) for a in idx["adj"]]), dtype=np.int32)
    if ids.size == 0:
        ids = np.zeros(1, np.int64)
        down = np.zeros(1, np.int64)
    keys_a = None if keys is None else np.ascontiguousarray(keys, dtype=np.uint64)
    out_ids = np.empty((max(nq, 1), stride), dtype=np.int64)
    out_d = np.empty((max(nq, 1), stride), dtype=np.float64)
    stats = np.zeros((max(nq, 1), 4), dtype=np.int64)
    lib().ho_search(_p(X, C.c_float), n, d, idx["metric"], L + 1, _p(sizes, C.c_int64),
                    _p(ids, C.c_int64), _p(down, C.c_int64), _p(adj, C.c_int32), Mmax,
                    _p(Q, C.c_float), nq, _p(kq, C.c_int32), _p(efq, C.c_int32), int(ef_upper), int(ef_l1),
                    int(descend_all), int(exact_upper),
                    idx["seed"] if seed is None else seed,
                    None if keys_a is None else _p(keys_a, C.c_uint64),
                    _p(out_ids, C.c_int64), _p(out_d, C.c_double), stride, _p(stats, C.c_int64))
    return out_ids[:nq], out_d[:nq], stats[:nq]


def greedy_layer(X, ids, adj, q, start, metric=L2):
    X, q = _f32(X), _f32(q)
    ids_a = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    hops = C.c_int64(0)
    evals = C.c_int64(0)
    r = lib().ho_greedy_layer(_p(X, C.c_float), X.shape[1], metric,
                              None if ids_a is None else _p(ids_a, C.c_int64), _p(adj, C.c_int32),
                              adj.shape[1], _p(q, C.c_float), start, C.byref(hops), C.byref(evals))
    return int(r), hops.value, evals.value


def bruteforce(X, Q, k, metric=L2):
    X, Q = _f32(X), _f32(Q)
    nq = Q.shape[0]
    ids = np.empty((max(nq, 1), k), dtype=np.int64)
    dd = np.empty((max(nq, 1), k), dtype=np.float64)
    lib().ho_bruteforce(_p(X, C.c_float), X.shape[0], X.shape[1], metric, _p(Q, C.c_float), nq, k,
                        _p(ids, C.c_int64), _p(dd, C.c_double))
    return ids[:nq], dd[:nq]


def bf16_bits(x: np.ndarray) -> np.ndarray:
    f = lib().ho_bf16_bits
    x = np.asarray(x, dtype=np.float32).reshape(-1)
    return np.array([f(float(v)) for v in x], dtype=np.uint16)


def e4m3_bits(x: np.ndarray) -> np.ndarray:
    f = lib().ho_e4m3_bits
    x = np.asarray(x, dtype=np.float32).reshape(-1)
    return np.array([f(v) for v in x.tolist()], dtype=np.uint8)


def e4m3_value(code: int) -> float:
    return lib().ho_e4m3_value(code)


def recall_at_k(found_ids, gt_ids, gt_d, found_d=None, k=None):
    """Recall@k (Sec. 2): |A_q ∩ O_q| / k per query.  A returned id also
    counts when its FP64 distance equals the k-th ground-truth distance
    (ties at the boundary)."""
    found_ids = np.asarray(found_ids)
    gt_ids = np.asarray(gt_ids)
    k = k or gt_ids.shape[1]
    out = np.empty(found_ids.shape[0])
    for q in range(found_ids.shape[0]):
        gt = set(gt_ids[q, :k].tolist())
        hits = 0
        for j in range(k):
            v = found_ids[q, j]
            if v in gt:
                hits += 1
            elif found_d is not None and v >= 0 and found_d[q, j] == gt_d[q, k - 1]:
                hits += 1
        out[q] = hits / k
    return out
