"""Pins of the FP64 oracle against facts fixed outside the oracle itself:
published generator outputs, closed forms, exhaustive enumeration of ring
ranges on tiny planar inputs, textbook brute force (scipy), invariants the
paper proves, and library conversions (torch) for the number formats.

Each test names the passage it pins.  No GPU is used.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ RNG

def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(l) for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_published_outputs():
    """The oracle's derive(h, j) is output j of SplitMix64 seeded with h."""
    want = _golden("splitmix64_seed1234567.txt")
    got = [O.derive(1234567, j) for j in range(len(want))]
    assert got == want
    # the input generator module implements the same published generator
    assert [int(v) for v in synth.splitmix64(1234567, 5)] == want


def test_bounded_is_uniform_chi2():
    """bounded(u, s) = floor(u s / 2^64) is uniform on [0, s) (chi-square)."""
    s, N = 37, 37 * 400
    h = O.derive(99, 7)
    counts = np.bincount([O.bounded(O.derive(h, j), s) for j in range(N)], minlength=s)
    exp = N / s
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # 36 degrees of freedom: P(chi2 > 70) < 1e-3
    assert chi2 < 70, chi2
    # exact small cases
    assert O.bounded(0, 10) == 0
    assert O.bounded(2**64 - 1, 10) == 9
    assert O.bounded(2**63, 10) == 5


# ----------------------------------------------- Alg. 2 sampling, Cor. 2

def test_sample_positions_sorted_distinct_subset():
    """Alg. 2 draws with replacement; the layer is the distinct set."""
    for s, t in [(1, 1), (5, 3), (1000, 63), (10000, 625)]:
        pos = O.sample_positions(3, 1, 0, s, t)
        assert np.all(np.diff(pos) > 0)
        assert pos.min() >= 0 and pos.max() < s
        assert 1 <= len(pos) <= min(s, t)


def test_sample_distinct_count_closed_form():
    """E[#distinct of t draws with replacement from s] = s (1 - (1 - 1/s)^t)."""
    s, t, trials = 2000, 125, 400
    cnt = np.array([len(O.sample_positions(11, 1, a, s, t)) for a in range(trials)], dtype=float)
    mean = s * (1 - (1 - 1 / s) ** t)
    # variance of the distinct count (occupancy problem)
    var = s * (1 - 1 / s) ** t + s * (s - 1) * (1 - 2 / s) ** t - (s * (1 - 1 / s) ** t) ** 2
    se = math.sqrt(var / trials)
    assert abs(cnt.mean() - mean) < 5 * se, (cnt.mean(), mean, se)


def test_order_rank_is_a_permutation():
    """The NSW insertion order is a permutation of 0..s-1 for every size."""
    for s in [1, 2, 3, 4, 5, 17, 64, 65, 1000, 4097]:
        r = O.order_ranks(5, 2, s)
        assert sorted(r.tolist()) == list(range(s))
    # different layers / seeds give different orders
    a, b = O.order_ranks(5, 2, 1000), O.order_ranks(5, 3, 1000)
    assert not np.array_equal(a, b)


def test_ring_window_definition():
    """Eq. 1 window: w - 1 <= eps(s) * s < w, eps = c0 d ln(s)/s 2^m;
    w = s + 1 (vacuous) once eps >= 1."""
    from fractions import Fraction

    for c0, d, s, m in [(1.0, 32, 10000, 4), (1.0, 128, 10**6, 4), (0.01, 32, 10000, 4), (1.0, 32, 600, 4),
                        (0.001, 2, 12, 1), (0.5, 3, 97, 2)]:
        w = O.ring_window(c0, d, s, m)
        es = c0 * d * math.log(s) * 2**m
        if es >= s:
            assert w == s + 1
        else:
            assert Fraction(w - 1) <= Fraction(es) < Fraction(w)


def test_ring_miss_rate_matches_sampling_probability():
    """A fixed window of w of the s points is missed by t draws with
    replacement with probability (1 - w/s)^t (the event the Las-Vegas loop
    of Alg. 2 retries on).  The oracle's sampled ring checks must miss at
    that rate."""
    rng = np.random.default_rng(0)
    s, t, d = 400, 25, 3
    X = rng.random((s, d)).astype(np.float32)
    prev = np.arange(s)
    w = 20
    r = 20
    misses = trials = 0
    for a in range(150):
        pos = O.sample_positions(7, 1, a, s, t)
        _, ok = O.verify(X, prev, pos, 7, 1, a, r, w)
        misses += int((~ok).sum())
        trials += r
    p = (1 - w / s) ** t
    se = math.sqrt(p * (1 - p) / trials)
    assert abs(misses / trials - p) < 5 * se, (misses / trials, p)


# ------------------------------------------ eps-nets of ring ranges (tiny)

def _data_centre_enumeration(X, prev_pos_net, w):
    """Independent check over every data-point centre and every window."""
    n = len(X)
    if w > n:
        return True
    D = ((X[:, None, :].astype(np.float64) - X[None, :, :].astype(np.float64)) ** 2).sum(-1)
    net = np.zeros(n, bool)
    net[prev_pos_net] = True
    for c in range(n):
        order = np.lexsort((np.arange(n), D[c]))
        vals = D[c][order]
        for a0 in range(0, n - w + 1):
            lo, hi = vals[a0], vals[a0 + w - 1]
            inside = (D[c] >= lo) & (D[c] <= hi)
            if not (inside & net).any():
                return False
    return True


def _plane_centres(P, rng):
    """Centres meeting every cell of the arrangement of perpendicular
    bisectors of a planar point set: around every vertex at the middle of
    each angle between incident lines, along every line on both sides, far
    away in many directions, the data points, and random points."""
    lines = []
    for i, j in itertools.combinations(range(len(P)), 2):
        a = 2.0 * (P[j] - P[i])
        b = float(P[j] @ P[j] - P[i] @ P[i])
        lines.append((a, b))
    scale = float(np.ptp(P)) + 1.0
    eps = 1e-6 * scale
    cs = [p for p in P]
    verts = []
    for (a1, b1), (a2, b2) in itertools.combinations(lines, 2):
        A = np.stack([a1, a2])
        if abs(np.linalg.det(A)) < 1e-12:
            continue
        verts.append(np.linalg.solve(A, np.array([b1, b2])))
    for v in verts:
        angs = []
        for a, b in lines:
            if abs(a @ v - b) < 1e-9 * scale * np.linalg.norm(a):
                t = math.atan2(-a[0], a[1])
                angs += [t % (2 * math.pi), (t + math.pi) % (2 * math.pi)]
        angs = sorted(set(angs)) or [0.0]
        for k in range(len(angs)):
            t0 = angs[k]
            t1 = angs[(k + 1) % len(angs)] + (2 * math.pi if k + 1 == len(angs) else 0.0)
            tm = 0.5 * (t0 + t1)
            cs.append(v + eps * np.array([math.cos(tm), math.sin(tm)]))
    for a, b in lines:
        nrm = a / np.linalg.norm(a)
        tang = np.array([-nrm[1], nrm[0]])
        base = nrm * (b / np.linalg.norm(a))
        for tpos in np.linspace(-3 * scale, 3 * scale, 41):
            for side in (-1, 1):
                cs.append(base + tpos * tang + side * eps * nrm)
    for t in np.linspace(0, 2 * math.pi, 720, endpoint=False):
        cs.append(1e4 * scale * np.array([math.cos(t), math.sin(t)]))
    cs += list(rng.uniform(P.min() - scale, P.max() + scale, size=(2000, 2)))
    return np.array(cs)


def _plane_enumeration(P, net_pos, w, centres):
    net = np.zeros(len(P), bool)
    net[net_pos] = True
    D = ((centres[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    order = np.argsort(D, axis=1, kind="stable")
    hit = net[order]  # per centre, net membership in distance order
    n = len(P)
    if w > n:
        return True
    # a window of w consecutive ranks without a net point = longest run > w-1
    run = np.zeros(len(centres), int)
    best = np.zeros(len(centres), int)
    for k in range(n):
        run = np.where(hit[:, k], 0, run + 1)
        best = np.maximum(best, run)
    return bool((best < w).all())


def test_epsnet_exhaustive_matches_enumeration():
    """Def. 2 ring ranges / App. B eps-net definition on tiny planar sets:
    (a) the oracle's exhaustive IsEpsNet over data centres equals an
    independent enumeration of every (centre, window);  (b) a set that is an
    eps-net for rings around every centre of the plane passes the oracle's
    check (its rings are a sub-family);  (c) a planted set that misses one
    heavy ring fails it."""
    rng = np.random.default_rng(1)
    agree = plane_nets = 0
    for trial in range(40):
        n = int(rng.integers(6, 12))
        P = rng.random((n, 2))
        X = P.astype(np.float32)
        Pd = X.astype(np.float64)
        w = int(rng.integers(2, n))
        k = int(rng.integers(1, n))
        net_pos = np.sort(rng.choice(n, size=k, replace=False))
        ok_oracle, _ = O.verify(X, np.arange(n), net_pos, 0, 1, 0, 1, w, exhaustive=True)
        ok_enum = _data_centre_enumeration(X, net_pos, w)
        assert ok_oracle == ok_enum, (trial, n, w, net_pos)
        agree += 1
        if _plane_enumeration(Pd, net_pos, w, _plane_centres(Pd, rng)):
            plane_nets += 1
            assert ok_oracle
    assert agree == 40 and plane_nets >= 1
    # planted miss: the w points nearest to point 0 (a ring around x_0) hold no net point
    P = rng.random((10, 2)).astype(np.float32)
    D = ((P - P[0]) ** 2).sum(1)
    near = np.argsort(D)[:4]
    net_pos = np.setdiff1d(np.arange(10), near)
    ok, _ = O.verify(P, np.arange(10), net_pos, 0, 1, 0, 1, 4, exhaustive=True)
    assert not ok


def test_sampled_rings_are_heavy_windows():
    """Each sampled ring (App. G: r random ranges) holds exactly w points,
    i.e. more than eps*s: its verdict equals a direct check of that window."""
    rng = np.random.default_rng(2)
    s, d, w, r = 300, 4, 17, 12
    X = rng.random((s, d)).astype(np.float32)
    pos = O.sample_positions(9, 1, 3, s, 40)
    _, ok = O.verify(X, np.arange(s), pos, 9, 1, 3, r, w)
    bc = O.derive(O.derive(O.derive(9, 0x5243454E), 1), 3)
    bs = O.derive(O.derive(O.derive(9, 0x52535441), 1), 3)
    D = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for q in range(r):
        c = O.bounded(O.derive(bc, q), s)
        a0 = O.bounded(O.derive(bs, q), s - w + 1)
        order = np.lexsort((np.arange(s), D[c]))
        window = set(order[a0:a0 + w].tolist())
        assert len(window) == w
        assert ok[q] == bool(window & set(pos.tolist()))


# --------------------------------------------- Alg. 1 layers, Lemma 1, Cor. 3

@pytest.mark.parametrize("n,d,m", [(10000, 32, 4), (3000, 8, 2), (500, 3, 3), (20, 2, 4), (15, 2, 4), (1, 2, 4)])
def test_layer_invariants(n, d, m):
    """Lemma 1: |L_i| <= ceil(|L_{i-1}| / 2^m); Def. 1: L_i subset of L_{i-1}
    with inter-layer edges between copies of a point; Cor. 3: L = O(log n /
    m); index size sum |L_i| = O(n) (Sec. 3.2)."""
    X = synth.uniform_cube(n, d, seed=4)
    idx = O.build_layers(X, m=m, seed=3)
    L = idx["L"]
    sizes = [len(a) for a in idx["ids"]]
    assert sizes[0] == n
    for i in range(1, L + 1):
        prev, cur, down = idx["ids"][i - 1], idx["ids"][i], idx["down"][i]
        assert sizes[i] <= -(-sizes[i - 1] // 2**m)
        assert sizes[i - 1] >= 2**m
        assert np.all(np.diff(cur) > 0)
        assert np.array_equal(prev[down], cur)
    if L > 0 or n >= 2**m:
        assert sizes[L] < 2**m or L == 63
    assert L <= math.ceil(math.log(max(n, 2)) / math.log(2**m)) + 1
    assert sum(sizes) <= n * 2**m / (2**m - 1) + L + 1


def test_las_vegas_retries_are_counted():
    """Alg. 2 repeats until IsEpsNet holds: with a small c0 (narrow heavy
    rings) several attempts are needed, and with max_attempts too small the
    build reports failure."""
    X = synth.uniform_cube(4000, 8, seed=5)
    idx = O.build_layers(X, c0=0.06, r=60, seed=1, max_attempts=2000)
    assert max(idx["attempts"]) >= 1
    with pytest.raises(RuntimeError):
        O.build_layers(X, c0=0.002, r=200, seed=1, max_attempts=2)


# ------------------------------------------------------- navigable graphs

def test_knn_graph_equals_bruteforce():
    """App. G knn graph: each point's list is its exact M nearest (scipy)."""
    X = synth.uniform_cube(500, 6, seed=6)
    ids = np.arange(500)
    fwd, fwd_d = O.forward_lists(X, ids, 0, 0, M=8, graph=O.GRAPH_KNN)
    D = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    np.fill_diagonal(D, np.inf)
    want = np.lexsort((np.tile(np.arange(500), (500, 1)), D), axis=1)[:, :8]
    assert np.array_equal(fwd, want)
    assert np.allclose(fwd_d, np.take_along_axis(D, want, 1), rtol=1e-12)


def test_nsw_forward_lists_are_nearest_predecessors():
    """App. B NSW: the point inserted at rank r links to its M nearest among
    the points inserted before it (brute force over predecessors)."""
    X = synth.uniform_cube(400, 5, seed=7)
    ids = np.arange(400)
    fwd, fwd_d = O.forward_lists(X, ids, 3, 0, M=6)
    rank = O.order_ranks(3, 0, 400)
    D = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for p in range(400):
        pred = np.where(rank < rank[p])[0]
        order = pred[np.lexsort((pred, D[p, pred]))][:6]
        got = fwd[p][fwd[p] >= 0]
        assert np.array_equal(got, order)
        assert len(got) == min(6, rank[p])


def test_edge_rule_properties():
    """Edge rule: the nearest predecessor first, then the nearest Mmax-1
    (by distance, index) of forward and reverse links; no duplicates; every
    point keeps a path to the first inserted point (connected graph)."""
    X = synth.uniform_cube(2000, 8, seed=8)
    ids = np.arange(2000)
    M, Mmax = 6, 10
    fwd, fwd_d = O.forward_lists(X, ids, 1, 0, M=M)
    adj = O.edge_rule(fwd, fwd_d, Mmax=Mmax)
    rank = O.order_ranks(1, 0, 2000)
    D = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    rev = [set() for _ in range(2000)]
    for p in range(2000):
        for v in fwd[p]:
            if v >= 0:
                rev[v].add(p)
    for v in range(2000):
        row = adj[v][adj[v] >= 0]
        assert len(set(row.tolist())) == len(row)
        cand = set(fwd[v][fwd[v] >= 0].tolist()) | rev[v]
        assert set(row.tolist()) <= cand
        if fwd[v][0] >= 0:
            assert row[0] == fwd[v][0]
            rest = row[1:]
            pool = sorted(cand - {int(fwd[v][0])}, key=lambda u: (D[v, u], u))
            assert rest.tolist() == pool[:Mmax - 1]
        else:
            assert rank[v] == 0
    # following the first entry reaches the first inserted point
    root = int(np.argmin(rank))
    for v in range(0, 2000, 37):
        u, steps = v, 0
        while u != root:
            u = int(adj[u][0])
            steps += 1
            assert steps < 2000
    import networkx as nx

    G = nx.Graph()
    G.add_nodes_from(range(2000))
    G.add_edges_from((v, int(u)) for v in range(2000) for u in adj[v] if u >= 0)
    assert nx.is_connected(G)


# ------------------------------------------------------------- queries

def test_complete_graph_greedy_is_exact():
    """App. B: the complete graph is navigable; GreedySearch (Alg. 4) on it
    returns the exact nearest neighbour from any start."""
    X = synth.uniform_cube(30, 4, seed=9)
    Q = synth.uniform_cube(50, 4, seed=10)
    idx = O.build_index(X, M=29, Mmax=32, m=4, seed=2)
    gt, _ = O.bruteforce(X, Q, 1)
    for qi in range(50):
        for start in [0, 7, 29]:
            c, hops, _ = O.greedy_layer(X, None, idx["adj"][0], Q[qi], start)
            assert c == gt[qi, 0]
    ids, _, _ = O.search(idx, X, Q, k=1, ef=1)
    assert np.array_equal(ids[:, 0], gt[:, 0])


def test_beam_covering_all_nodes_is_exact_knn():
    """A beam as wide as the layer, on a graph where every node is reachable
    from every other, returns the exact k nearest (Sec. 2 k-NN query)."""
    import networkx as nx

    X = synth.uniform_cube(300, 6, seed=11)
    Q = synth.uniform_cube(40, 6, seed=12)
    idx = O.build_index(X, seed=4)
    G = nx.DiGraph()
    G.add_edges_from((v, int(u)) for v in range(300) for u in idx["adj"][0][v] if u >= 0)
    assert nx.is_strongly_connected(G)
    gi, gd = O.bruteforce(X, Q, 10)
    ids, dd, _ = O.search(idx, X, Q, k=10, ef=300)
    assert np.array_equal(ids, gi)
    assert np.allclose(dd, gd, rtol=1e-12)


def test_beam_width_one_is_greedy():
    """With ef = 1 and k = 1 the beam is GreedySearch of Alg. 4."""
    X = synth.uniform_cube(2000, 8, seed=13)
    Q = synth.uniform_cube(100, 8, seed=14)
    idx = O.build_index(X, seed=5, max_layers=0)
    # no upper layers: the entry is drawn on layer 0 directly
    idx1 = O.build_index(X, seed=5, max_layers=1)
    for ix in (idx, idx1):
        ids, _, st = O.search(ix, X, Q, k=1, ef=1)
        for q in range(100):
            e = int(st[q, 3])
            if ix["L"] == 0:
                c, _, _ = O.greedy_layer(X, None, ix["adj"][0], Q[q], e)
                assert ids[q, 0] == c


def test_greedy_hop_bound():
    """Proof of Thm. 1: each greedy move is strictly closer to q, so the
    number of moves is at most the number of points strictly closer than
    the start."""
    X = synth.uniform_cube(3000, 8, seed=15)
    Q = synth.uniform_cube(60, 8, seed=16)
    idx = O.build_index(X, seed=6)
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    rng = np.random.default_rng(3)
    for q in range(60):
        start = int(rng.integers(0, 3000))
        c, hops, _ = O.greedy_layer(X, None, idx["adj"][0], Q[q], start)
        assert hops <= int((D[q] < D[q, start]).sum())
        assert D[q, c] <= D[q, start]


def test_query_evaluations_grow_polylog():
    """Thm. 1: query time O(d d* rho log^2 n).  Distance evaluations per
    query, for n = 2^10 .. 2^14 (exponential coordinates, App. G), must fit
    a log^2 n law better than a linear one.  The constant is not pinned (the
    paper gives none)."""
    ns = [2**10, 2**11, 2**12, 2**13, 2**14]
    ev = []
    for n in ns:
        X = synth.exponential(n, 16, 4.0, seed=20)
        Q = synth.exponential(200, 16, 4.0, seed=21)
        idx = O.build_index(X, seed=7)
        _, _, st = O.search(idx, X, Q, k=10, ef=32)
        ev.append(st[:, 0].mean())
    ev = np.array(ev)
    lg2 = np.log(ns) ** 2
    A = np.stack([lg2, np.ones(5)], 1)
    r_log = np.linalg.lstsq(A, ev, rcond=None)[1]
    B = np.stack([np.array(ns, float), np.ones(5)], 1)
    r_lin = np.linalg.lstsq(B, ev, rcond=None)[1]
    assert r_log[0] < r_lin[0], (ev, r_log, r_lin)
    assert ev[-1] / ev[0] < 16 / 4, ev


def test_recall_definition():
    """Recall@k = |A_q intersect O_q| / k (Sec. 2)."""
    gt = np.array([[1, 2, 3, 4]])
    gd = np.array([[0.1, 0.2, 0.3, 0.4]])
    assert O.recall_at_k(np.array([[1, 2, 3, 4]]), gt, gd)[0] == 1.0
    assert O.recall_at_k(np.array([[4, 9, 1, 8]]), gt, gd)[0] == 0.5
    # a tie with the k-th distance counts
    assert O.recall_at_k(np.array([[1, 2, 3, 7]]), gt, gd, np.array([[0.1, 0.2, 0.3, 0.4]]))[0] == 1.0


def test_search_exact_on_tiny_index():
    """Edge cases: n smaller than 2^m (no upper layer), k > n (padding)."""
    X = synth.uniform_cube(9, 3, seed=17)
    Q = synth.uniform_cube(5, 3, seed=18)
    idx = O.build_index(X, seed=1)
    assert idx["L"] == 0
    ids, dd, _ = O.search(idx, X, Q, k=12, ef=20)
    gi, gd = O.bruteforce(X, Q, 9)
    assert np.array_equal(ids[:, :9], gi)
    assert np.all(ids[:, 9:] == -1) and np.all(np.isinf(dd[:, 9:]))


def test_angular_distance_definition():
    """App. G: angular distance 1 - cos, equal to |x/|x| - y/|y||^2 / 2."""
    rng = np.random.default_rng(4)
    a, b = rng.normal(size=8).astype(np.float32), rng.normal(size=8).astype(np.float32)
    v = O.dist(a, b, O.ANGULAR)
    an, bn = a / np.linalg.norm(a.astype(np.float64)), b / np.linalg.norm(b.astype(np.float64))
    assert abs(v - 0.5 * ((an - bn) ** 2).sum()) < 1e-12
    assert abs(v - (1 - 1 + cdist(a[None].astype(np.float64), b[None].astype(np.float64), "cosine")[0, 0])) < 1e-12


# ------------------------------------------------------ number formats

def test_bf16_rounding_matches_library():
    """Round-to-nearest-even float32 -> bfloat16 (format definition) agrees
    with torch's conversion on representable values, midpoints (ties) and
    random floats."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    vals = []
    hi16 = rng.integers(0, 2**16, size=3000, dtype=np.uint32)
    for h in hi16:
        for low in (0, 0x8000, 0x7FFF, 0x8001, 0x1234):
            vals.append((int(h) << 16) | low)
    vals += [0x7F7FFFFF, 0x7F7F8000, 0x00000001, 0x80000001]
    x = np.array(vals, dtype=np.uint32).view(np.float32)
    x = x[np.isfinite(x)]
    mine = O.bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(mine, ref)


def test_e4m3_rounding_matches_library():
    """OCP E4M3: all 256 codes decode as torch's float8_e4m3fn; encoding
    (round to nearest even) agrees with torch for |x| <= 448, and larger
    magnitudes saturate to 448 as the satfinite rule of the format says."""
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    mine = np.array([O.e4m3_value(int(c)) for c in codes])
    assert np.array_equal(np.isnan(mine), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.array_equal(mine[ok], ref[ok])
    rng = np.random.default_rng(6)
    finite = ref[ok & (np.abs(ref) <= 448)]
    mids = (np.sort(np.unique(finite))[:-1] + np.sort(np.unique(finite))[1:]) / 2
    x = np.concatenate([finite, mids, rng.normal(scale=50, size=4000),
                        rng.uniform(-448, 448, 4000), np.ldexp(rng.uniform(-1, 1, 2000), -8)]).astype(np.float32)
    x = x[np.abs(x) <= 448]
    mine = O.e4m3_bits(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(mine, ref)
    big = np.array([448.5, 449, 460, 480, 1e6, np.inf, -500], dtype=np.float32)
    codes = O.e4m3_bits(big)
    assert all(abs(O.e4m3_value(int(c))) == 448 for c in codes)


# ------------------------------------------------ Alg. 3 halving sampler

def test_halving_sizes_and_pairs():
    """BuildEpsNetDiscV2 (Alg. 3): each halving step keeps exactly one point
    of every matched pair (here consecutive list entries) and the unmatched
    last one, so m steps leave ceil-halved m times; survivors are sorted."""
    for s in [1, 2, 3, 17, 100, 1023, 4096]:
        for m in [1, 2, 4]:
            want = s
            for _ in range(m):
                want = (want + 1) // 2
            p = O.halving_positions(s, m, seed=5, layer=1)
            assert len(p) == want
            assert np.all(np.diff(p) > 0)
    p = O.halving_positions(101, 1, seed=9, layer=2)
    assert [int(v) // 2 for v in p] == list(range(51))  # one of (2j, 2j+1), and 100 unmatched
    assert p[-1] == 100


def test_halving_survival_is_uniform():
    """Every point survives m steps with probability 2^-m: over 4000 seeds,
    each of 64 positions survives 2 steps about 1000 times (binomial, 6 sd)."""
    counts = np.zeros(64)
    for seed in range(4000):
        counts[O.halving_positions(64, 2, seed=seed, layer=1)] += 1
    assert counts.sum() == 4000 * 16
    sd = math.sqrt(4000 * 0.25 * 0.75)
    assert np.all(np.abs(counts - 1000) < 6 * sd)


def test_halving_layers_ignore_values():
    """The halving hierarchy depends on sizes and the seed only: two point
    sets of the same size get the same layers, |L_i| halves m times per
    layer, and down pointers index the layer below."""
    X1 = synth.uniform_cube(5000, 8, seed=1)
    X2 = synth.gaussian_mixture(5000, 8, 10, seed=2)[0]
    a = O.build_layers(X1, m=3, seed=4, sampler=O.SAMPLER_HALVING)
    b = O.build_layers(X2, m=3, seed=4, sampler=O.SAMPLER_HALVING)
    assert a["L"] == b["L"] and all(np.array_equal(u, v) for u, v in zip(a["ids"], b["ids"]))
    for i in range(1, a["L"] + 1):
        prev = a["ids"][i - 1]
        assert np.array_equal(prev[a["down"][i]], a["ids"][i])
        want = len(prev)
        for _ in range(3):
            want = (want + 1) // 2
        assert len(a["ids"][i]) == want


def test_exact_upper_layers_pick_true_nearest():
    """With exact_upper covering the upper layers, layer 1 hands layer 0 the
    copy of the query's true nearest layer-1 point (scipy brute force), and
    a width-1 search on layer 0 is GreedySearch from there (Alg. 4)."""
    X = synth.uniform_cube(3000, 8, seed=21)
    Q = synth.uniform_cube(60, 8, seed=22)
    idx = O.build_index(X, seed=5)
    ids1 = idx["ids"][1]
    near1 = np.argmin(cdist(Q.astype(np.float64), X[ids1].astype(np.float64), "sqeuclidean"), axis=1)
    start0 = idx["down"][1][near1]
    got, _, st = O.search(idx, X, Q, k=1, ef=1, ef_upper=1, exact_upper=10**9)
    for q in range(len(Q)):
        want, _, _ = O.greedy_layer(X, None, idx["adj"][0], Q[q], int(start0[q]))
        assert got[q, 0] == want
    # every upper-layer point is evaluated once per query
    assert np.all(st[:, 0] >= sum(len(a) for a in idx["ids"][1:]))


# ------------------------------------------------ dynamic insert (App. C)

def test_insert_forward_rows_and_structure():
    """Insert (App. C): an inserted point's forward list in each layer it
    joins is its exact M nearest current members (scipy brute force, ties by
    position); layers stay ascending with consistent down pointers; a
    search for an inserted point finds it at distance 0."""
    X = synth.uniform_cube(2600, 6, seed=31)
    idx = O.build_index(X[:2000], seed=7)
    M = idx["M"]
    new = np.arange(2000, 2600)
    before = [a.copy() for a in idx["ids"]]
    O.insert(idx, X, new)
    for i in range(idx["L"] + 1):
        ids = idx["ids"][i]
        assert np.all(np.diff(ids) > 0)
        if i >= 1:
            assert np.array_equal(idx["ids"][i - 1][idx["down"][i]], ids)
        for pos in range(len(before[i]), len(ids)):
            p = ids[pos]
            d = cdist(X[p:p + 1].astype(np.float64), X[ids[:pos]].astype(np.float64), "sqeuclidean")[0]
            want = np.lexsort((np.arange(pos), d))[:M]
            assert np.array_equal(idx["fwd"][i][pos][:len(want)], want)
    got, dist, _ = O.search(idx, X, X[new[::50]], k=1, ef=64)
    assert np.array_equal(got[:, 0], new[::50]) and np.all(dist[:, 0] == 0)


def test_insert_promotion_rate():
    """An inserted point joins layer i with probability 2^-m given layer
    i-1 (the built layers' rate): about 1/16 of 20000 ids reach layer 1."""
    hits = sum(1 for p in range(20000) if len(O.insert_layers(3, p, 4, 5)) > 1)
    sd = math.sqrt(20000 / 16 * 15 / 16)
    assert abs(hits - 20000 / 16) < 6 * sd
    deep = [O.insert_layers(3, p, 2, 6) for p in range(4000)]
    assert all(v == list(range(len(v))) for v in deep)


def test_delete_tombstones_give_live_nearest():
    """Delete (App. C) as tombstones: with a beam covering the whole base
    layer the result is the exact k nearest live points (scipy)."""
    X = synth.uniform_cube(400, 5, seed=51)
    Q = synth.uniform_cube(30, 5, seed=52)
    idx = O.build_index(X, seed=8)
    dead = np.zeros(len(X), bool)
    dead[::3] = True
    got, gd, _ = O.search(idx, X, Q, k=10, ef=400, deleted=dead)
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    D[:, dead] = np.inf
    want = np.argsort(D, axis=1, kind="stable")[:, :10]
    assert np.array_equal(got, want)
    assert not dead[got].any()


# ------------------------------- upper-layer candidate sets (Sec. 2.2)
#
# Sec. 2.2 keeps "a set of candidates at each step" on the way down.  The
# pins below remove the edges of the layers under the one being checked, so
# that those layers' beams can only return what they were seeded with:
# the search's output is then exactly the hand-down of the checked layer,
# and scipy brute force over that layer's points fixes it.  A wrong down
# array, unsorted seeds, or truncation to the wrong width fails them.

def _edgeless(idx, layers):
    """Copy of idx whose listed layers have no edges (every row -1)."""
    out = dict(idx)
    out["adj"] = [np.full_like(a, -1) if i in layers else a for i, a in enumerate(idx["adj"])]
    return out


def _strongly_connected(adj):
    import networkx as nx

    G = nx.DiGraph()
    G.add_nodes_from(range(len(adj)))
    G.add_edges_from((v, int(u)) for v in range(len(adj)) for u in adj[v] if u >= 0)
    return nx.is_strongly_connected(G)


def _nearest_of_layer(X, Q, ids, width):
    """The `width` points of a layer nearest to each query, ties by
    position, as global ids (scipy)."""
    D = cdist(Q.astype(np.float64), X[ids].astype(np.float64), "sqeuclidean")
    pos = np.array([np.lexsort((np.arange(len(ids)), D[q]))[:width] for q in range(len(Q))])
    return ids[pos]


@pytest.fixture(scope="module")
def hier3k():
    X = synth.uniform_cube(3000, 8, seed=41)
    Q = synth.uniform_cube(40, 8, seed=42)
    idx = O.build_index(X, seed=9)
    assert idx["L"] >= 2
    return X, Q, idx


def test_covering_beam_on_layer1_hands_down_its_nearest_set(hier3k):
    """A beam of width >= |L_1| on a strongly connected layer-1 graph
    evaluates the whole layer; with descend_all its candidates, sorted,
    seed layer 0, whose width-ef beam keeps the first ef.  Layer 0 without
    edges returns those seeds: the ef nearest layer-1 points (global ids)."""
    X, Q, idx = hier3k
    s1 = len(idx["ids"][1])
    assert _strongly_connected(idx["adj"][1])
    ix = _edgeless(idx, {0})
    for ef in (1, 7, 30):
        got, gd, st = O.search(ix, X, Q, k=ef, ef=ef, ef_upper=s1 + 5, descend_all=1)
        want = _nearest_of_layer(X, Q, idx["ids"][1], ef)
        assert np.array_equal(got, want), ef
        # the layer-0 candidate set starts as the first ef seeds: an edgeless
        # layer expands each of them once and nothing else
        assert np.all(st[:, 1] == ef), ef
        D = cdist(Q.astype(np.float64), X.astype(np.float64), "euclidean")
        assert np.allclose(gd, np.take_along_axis(D, want, 1), rtol=1e-12)


def test_best_candidate_only_without_descend_all(hier3k):
    """Without descend_all only the best candidate of the layer-1 beam goes
    down (Alg. 4 hands one node to the layer below): with edgeless layer 0
    the answer is the single nearest layer-1 point, padded."""
    X, Q, idx = hier3k
    s1 = len(idx["ids"][1])
    ix = _edgeless(idx, {0})
    got, gd, _ = O.search(ix, X, Q, k=3, ef=3, ef_upper=s1 + 5, descend_all=0)
    want = _nearest_of_layer(X, Q, idx["ids"][1], 1)
    assert np.array_equal(got[:, :1], want)
    assert np.all(got[:, 1:] == -1) and np.all(np.isinf(gd[:, 1:]))


def test_two_layer_hand_down_and_ef_l1(hier3k):
    """Layer 2 searched by a covering beam (ef_upper), layer 1 by a beam of
    width ef_l1 without edges: it keeps the first ef_l1 seeds from layer 2,
    which go down through both down arrays to edgeless layer 0.  The answer
    is the ef_l1 nearest layer-2 points, as global ids."""
    X, Q, idx = hier3k
    s2 = len(idx["ids"][2])
    assert _strongly_connected(idx["adj"][2])
    ix = _edgeless(idx, {0, 1})
    assert idx["L"] == 2  # layer 2 is the top: its beam starts at the entry
    for l1 in (1, 3, min(6, s2)):
        got, _, st = O.search(ix, X, Q, k=l1, ef=l1, ef_upper=s2 + 3, ef_l1=l1, descend_all=1)
        assert np.array_equal(got, _nearest_of_layer(X, Q, idx["ids"][2], l1)), l1
        # a beam wider than its layer never fills, so it expands every node
        # of the connected layer 2; the edgeless layer-1 beam expands its l1
        # seeds (width 1 is GreedySearch instead, which makes no move there)
        assert np.all(st[:, 2] == s2 + (l1 if l1 > 1 else 0)), l1
    # ef_l1 = 0 falls back to ef_upper on layer 1: all of layer 2 goes down
    got, _, _ = O.search(ix, X, Q, k=s2, ef=s2, ef_upper=s2 + 3, ef_l1=0, descend_all=1)
    assert np.array_equal(got, _nearest_of_layer(X, Q, idx["ids"][2], s2))


def test_exact_sets_equal_covering_beams(hier3k):
    """Reading of Sec. 2.2 for small layers: the exact candidate set of a
    layer (exact_upper) is what a covering beam returns on a connected
    layer, so the two searches agree query by query, and both equal the
    brute-force hand-down on an edgeless layer 0."""
    X, Q, idx = hier3k
    s1 = len(idx["ids"][1])
    for ix in (idx, _edgeless(idx, {0})):
        a, ad, _ = O.search(ix, X, Q, k=10, ef=24, ef_upper=s1 + 5, descend_all=1)
        b, bd, _ = O.search(ix, X, Q, k=10, ef=24, ef_upper=s1 + 5, descend_all=1, exact_upper=s1)
        assert np.array_equal(a, b) and np.array_equal(ad, bd)


def test_greedy_upper_layers_chain_alg4(hier3k):
    """ef_upper = 1 is Alg. 4: GreedySearch on each layer from the copy of
    the previous result, starting at the reported entry node of the top
    layer; with k = ef = 1 the answer is the end of the layer-0 walk."""
    X, Q, idx = hier3k
    L = idx["L"]
    got, _, st = O.search(idx, X, Q, k=1, ef=1, ef_upper=1)
    for q in range(len(Q)):
        cur = int(st[q, 3])
        assert 0 <= cur < len(idx["ids"][L])
        for i in range(L, 0, -1):
            cur, _, _ = O.greedy_layer(X, idx["ids"][i], idx["adj"][i], Q[q], cur)
            cur = int(idx["down"][i][cur])
        end, _, _ = O.greedy_layer(X, None, idx["adj"][0], Q[q], cur)
        assert got[q, 0] == end
    # the entry node is uniform over the top layer's keys (Alg. 4: random root)
    many = synth.uniform_cube(4000, 8, seed=43)
    _, _, st = O.search(idx, X, many, k=1, ef=1)
    counts = np.bincount(st[:, 3], minlength=len(idx["ids"][L]))
    assert counts.min() > 0


# --------------------------------- delete with resampling (App. C, Delete)

def test_rebuild_from_a_layer_reproduces_the_build():
    """Building from layer i on top of the unchanged layer i - 1 draws the
    same random streams as the full build (Alg. 1 + Alg. 2): the same layers."""
    X = synth.uniform_cube(5000, 8, seed=62)
    idx = O.build_index(X, seed=4)
    for i in range(1, idx["L"] + 1):
        ids, down, att = O.build_layers_from(X, idx["ids"][i - 1], i, seed=4)
        assert len(ids) == idx["L"] - i + 1
        for j, (a, b) in enumerate(zip(ids, down)):
            assert np.array_equal(a, idx["ids"][i + j]) and np.array_equal(b, idx["down"][i + j])
            assert att[j] == idx["attempts"][i + j]


def test_delete_resamples_a_shrunken_layer_and_rebuilds_above():
    """App. C, Delete: a few deletions leave the layers as they are; once
    the live part of layer 1 falls below half of a fresh sample of the live
    points below, layer 1 is resampled from the live points of layer 0 and
    everything above is rebuilt: nested layers of live points, down pointers
    into the layer below, sizes within Lemma 1's bound."""
    X = synth.uniform_cube(6000, 8, seed=63)
    idx = O.build_index(X, seed=5)
    before = [a.copy() for a in idx["ids"]]
    dead = np.zeros(len(X), bool)
    dead[before[1][:5]] = True
    assert O.delete(idx, X, dead) is None
    assert all(np.array_equal(a, b) for a, b in zip(idx["ids"], before))
    dead[before[1][: (2 * len(before[1])) // 3]] = True
    assert O.delete(idx, X, dead) == 1
    assert np.array_equal(idx["ids"][0], np.arange(len(X)))
    for i in range(1, idx["L"] + 1):
        ids, below = idx["ids"][i], idx["ids"][i - 1]
        assert not dead[ids].any()
        assert np.array_equal(below[idx["down"][i]], ids) and np.all(np.diff(ids) > 0)
        live_below = (~dead[below]).sum()
        assert len(ids) <= -(-live_below // 16)
        assert idx["adj"][i].shape == (len(ids), idx["Mmax"])
    # the rebuilt layer 1 is what a fresh build on the live points draws for layer 1
    fresh, _, _ = O.build_layers_from(X, np.nonzero(~dead)[0], 1, seed=5)
    assert np.array_equal(fresh[0], idx["ids"][1])


def test_search_after_resampling_is_exact_with_a_covering_beam():
    """After a resampling delete, a beam covering the base layer returns the
    exact k nearest live points (scipy), deleted ones never."""
    X = synth.uniform_cube(600, 5, seed=64)
    Q = synth.uniform_cube(30, 5, seed=65)
    idx = O.build_index(X, seed=6)
    dead = np.zeros(len(X), bool)
    dead[idx["ids"][1][: (2 * len(idx["ids"][1])) // 3]] = True
    dead[::7] = True
    assert O.delete(idx, X, dead) == 1
    got, _, _ = O.search(idx, X, Q, k=10, ef=600, deleted=dead)
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    D[:, dead] = np.inf
    assert np.array_equal(got, np.argsort(D, axis=1, kind="stable")[:, :10])
