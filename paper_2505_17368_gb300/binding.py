"""Thin ctypes binding of libhenn (include/henn.h): argument marshalling only.

Every step of index construction and search runs in the library's CUDA
kernels; this module converts arrays to pointers, fills the parameter
structs and raises on a non-OK status.  There is no fallback: if the
compiled library is missing, loading fails with an error.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA).  PyTorch
is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhenn.so")

L2, ANGULAR = 0, 1
F32, BF16, FP8E4M3 = 0, 1, 2
GRAPH_NSW, GRAPH_KNN = 0, 1
TILES_AUTO, TILES_SIMT, TILES_TCGEN05 = 0, 1, 2
SAMPLER_SAMPLING, SAMPLER_HALVING = 0, 1
EXACT_SORT, EXACT_TILES, EXACT_SCAN = 0, 1, 2
MAX_LAYERS = 32

STATUS = {
    0: "HENN_OK",
    1: "HENN_ERR_INVALID_ARG",
    2: "HENN_ERR_OOM",
    3: "HENN_ERR_CUDA",
    4: "HENN_ERR_EPSNET_NOT_FOUND",
    5: "HENN_ERR_TIMEOUT",
    6: "HENN_ERR_UNSUPPORTED",
    7: "HENN_ERR_BUSY",
}
BUSY = 7

EXPORTS = [
    "henn_build_params_default",
    "henn_build",
    "henn_free",
    "henn_search_params_default",
    "henn_search",
    "henn_index_get_info",
    "henn_index_get_layer",
    "henn_exact_knn",
    "henn_greedy_probe",
    "henn_insert",
    "henn_delete",
    "henn_quantize_rows",
    "henn_last_error",
    "henn_serve_params_default",
    "henn_serve_create",
    "henn_serve_submit",
    "henn_serve_poll",
    "henn_serve_destroy",
    "henn_search_host_noalloc",
    "henn_last_search_ms",
]


class HennError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check_rows(Q, d):
    """Queries must be a 2-D array of rows of the index's dimension: the
    library reads nq * d floats from the buffer."""
    if len(Q.shape) != 2 or Q.shape[1] != d:
        raise HennError(1, f"queries must be a 2-D array of shape (nq, {d}), got {tuple(Q.shape)}")


class BuildParams(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32),
        ("metric", C.c_int32),
        ("storage", C.c_int32),
        ("graph", C.c_int32),
        ("m", C.c_int32),
        ("max_layers", C.c_int32),
        ("eps_c0", C.c_double),
        ("num_ranges", C.c_int32),
        ("max_attempts", C.c_int32),
        ("M", C.c_int32),
        ("Mmax", C.c_int32),
        ("tiles", C.c_int32),
        ("seed", C.c_uint64),
        ("sampler", C.c_int32),
        ("resample_share", C.c_double),
    ]


class SearchParams(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32),
        ("k", C.c_void_p),
        ("ef", C.c_void_p),
        ("k_uniform", C.c_int32),
        ("ef_uniform", C.c_int32),
        ("rerank_mult", C.c_int32),
        ("query_keys", C.c_void_p),
        ("stats", C.c_void_p),
        ("warps_per_block", C.c_int32),
        ("hash_bits", C.c_int32),
        ("ef_upper", C.c_int32),
        ("descend_all", C.c_int32),
        ("ef_l1", C.c_int32),
        ("exact_upper", C.c_int32),
        ("exact_method", C.c_int32),
        ("time_kernel", C.c_int32),
        ("team_size", C.c_int32),
        ("tile_n", C.c_int32),
    ]


class ServeParams(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32),
        ("ring_rows", C.c_int32),
        ("max_requests", C.c_int32),
        ("max_k", C.c_int32),
        ("max_ef", C.c_int32),
        ("ef_upper", C.c_int32),
        ("descend_all", C.c_int32),
        ("rerank_mult", C.c_int32),
        ("idle_ms", C.c_int32),
        ("ef_l1", C.c_int32),
        ("exact_upper", C.c_int32),
    ]


class IndexInfo(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32),
        ("n", C.c_int64),
        ("d", C.c_int32),
        ("metric", C.c_int32),
        ("storage", C.c_int32),
        ("graph", C.c_int32),
        ("M", C.c_int32),
        ("Mmax", C.c_int32),
        ("L", C.c_int32),
        ("sizes", C.c_int64 * MAX_LAYERS),
        ("attempts", C.c_int32 * MAX_LAYERS),
        ("ambiguous_rings", C.c_int32 * MAX_LAYERS),
        ("device_bytes", C.c_int64),
        ("uncertified_rows", C.c_int64),
        ("build_seconds", C.c_double),
        ("tile_seconds", C.c_double),
        ("tile_flops", C.c_double),
        ("tile_engine", C.c_int32),
        ("graph_instantiations", C.c_int32),
        ("graph_updates", C.c_int32),
    ]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libhenn.  Raises if the compiled library is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(
                f"libhenn is not built ({p} missing): run `python -c 'import __graft_entry__ as g; g.build()'`"
            )
        L = C.CDLL(p)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.henn_build_params_default.argtypes = [C.POINTER(BuildParams)]
        L.henn_build_params_default.restype = None
        L.henn_build.argtypes = [vp, i64, i32, i32, C.POINTER(BuildParams), vp, C.POINTER(vp)]
        L.henn_build.restype = i32
        L.henn_free.argtypes = [vp]
        L.henn_free.restype = None
        L.henn_search_params_default.argtypes = [C.POINTER(SearchParams)]
        L.henn_search_params_default.restype = None
        L.henn_search.argtypes = [vp, vp, i64, i32, C.POINTER(SearchParams), vp, vp, i32, vp]
        L.henn_search.restype = i32
        L.henn_index_get_info.argtypes = [vp, C.POINTER(IndexInfo)]
        L.henn_index_get_info.restype = i32
        L.henn_index_get_layer.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.henn_index_get_layer.restype = i32
        L.henn_exact_knn.argtypes = [vp, i64, i32, vp, i64, i32, i32, vp, vp, vp]
        L.henn_exact_knn.restype = i32
        L.henn_greedy_probe.argtypes = [vp, i32, vp, i64, vp, i32, vp, vp, vp, vp]
        L.henn_greedy_probe.restype = i32
        L.henn_insert.argtypes = [vp, vp, i64, i32, vp]
        L.henn_insert.restype = i32
        L.henn_delete.argtypes = [vp, vp, i64, vp]
        L.henn_delete.restype = i32
        L.henn_quantize_rows.argtypes = [vp, i64, i32, i32, vp, vp, vp]
        L.henn_quantize_rows.restype = i32
        L.henn_serve_params_default.argtypes = [C.POINTER(ServeParams)]
        L.henn_serve_params_default.restype = None
        L.henn_serve_create.argtypes = [vp, C.POINTER(ServeParams), C.POINTER(vp)]
        L.henn_serve_create.restype = i32
        L.henn_serve_submit.argtypes = [vp, vp, i32, i32, i32, vp, C.POINTER(i64)]
        L.henn_serve_submit.restype = i32
        L.henn_serve_poll.argtypes = [vp, i64, C.POINTER(i32), vp, vp]
        L.henn_serve_poll.restype = i32
        L.henn_serve_destroy.argtypes = [vp]
        L.henn_serve_destroy.restype = None
        L.henn_search_host_noalloc.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, i32, vp]
        L.henn_search_host_noalloc.restype = i32
        L.henn_last_search_ms.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(i32)]
        L.henn_last_search_ms.restype = i32
        L.henn_last_error.argtypes = []
        L.henn_last_error.restype = C.c_char_p
        _lib = L
        return L


def _check(status: int):
    if status != 0:
        raise HennError(status, load().henn_last_error().decode())


# ------------------------------------------------------------ marshalling

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, False, None
    if _is_torch(x):
        if not x.is_contiguous():
            x = x.contiguous()
        return C.c_void_p(x.data_ptr()), bool(x.is_cuda), x
    a = np.ascontiguousarray(x)
    return C.c_void_p(a.ctypes.data), False, a


def _stream(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class Index:
    """A HENN index resident in device memory (henn_build / henn_free)."""

    def __init__(self, X, metric=L2, storage=F32, graph=GRAPH_NSW, m=4, max_layers=0, eps_c0=1.0,
                 num_ranges=100, max_attempts=64, M=16, Mmax=32, tiles=TILES_AUTO, seed=0, stream=None,
                 sampler=SAMPLER_SAMPLING, resample_share=0.5):
        L = load()
        p = BuildParams()
        L.henn_build_params_default(C.byref(p))
        p.metric, p.storage, p.graph = metric, storage, graph
        p.m, p.max_layers, p.eps_c0 = m, max_layers, float(eps_c0)
        p.num_ranges, p.max_attempts, p.M, p.Mmax, p.tiles = num_ranges, max_attempts, M, Mmax, tiles
        p.seed = seed & 0xFFFFFFFFFFFFFFFF
        p.sampler = int(sampler)
        p.resample_share = float(resample_share)
        if _is_torch(X):
            import torch

            X = X.to(torch.float32)
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
        n, d = X.shape
        xp, on_dev, keep = _ptr(X)
        h = C.c_void_p()
        _check(L.henn_build(xp, n, d, int(on_dev), C.byref(p), _stream(stream), C.byref(h)))
        self._h = h
        self.n, self.d, self.M, self.Mmax = n, d, M, Mmax
        self.metric, self.storage = metric, storage
        del keep

    def insert(self, X, stream=None):
        """henn_insert: append the rows of X (n_new x d, host or CUDA) to the
        index; they get ids n, n + 1, ...  Returns the first new id."""
        if _is_torch(X):
            import torch

            X = X.to(torch.float32).contiguous()
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
        xp, on_dev, keep = _ptr(X)
        first = self.n
        _check(load().henn_insert(self._h, xp, X.shape[0], int(on_dev), _stream(stream)))
        self.n += X.shape[0]
        del keep
        return first

    def delete(self, ids, stream=None):
        """henn_delete: tombstone the points with these global ids, and
        resample and rebuild the upper layers when one has shrunk too far
        (App. C)."""
        ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64).reshape(-1))
        _check(load().henn_delete(self._h, C.c_void_p(ids.ctypes.data), ids.size, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().henn_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = IndexInfo()
        inf.struct_size = C.sizeof(IndexInfo)
        _check(load().henn_index_get_info(self._h, C.byref(inf)))
        Lc = inf.L
        return dict(
            n=inf.n, d=inf.d, L=Lc, sizes=[inf.sizes[i] for i in range(Lc + 1)],
            attempts=[inf.attempts[i] for i in range(Lc + 1)],
            ambiguous_rings=[inf.ambiguous_rings[i] for i in range(Lc + 1)],
            device_bytes=inf.device_bytes, uncertified_rows=inf.uncertified_rows,
            build_seconds=inf.build_seconds, M=inf.M, Mmax=inf.Mmax, tile_seconds=inf.tile_seconds,
            tile_flops=inf.tile_flops, tile_engine=inf.tile_engine,
            graph_instantiations=inf.graph_instantiations, graph_updates=inf.graph_updates,
        )

    def layer(self, i: int) -> dict:
        s = self.info()["sizes"][i]
        ids = np.empty(s, np.int32)
        down = np.empty(s, np.int32)
        adj = np.empty((s, self.Mmax), np.int32)
        fwd = np.empty((s, self.M), np.int32)
        fwd_d = np.empty((s, self.M), np.float32)
        P = lambda a: C.c_void_p(a.ctypes.data)  # noqa: E731
        _check(load().henn_index_get_layer(self._h, i, P(ids), P(down), P(adj), P(fwd), P(fwd_d)))
        return dict(ids=ids, down=down, adj=adj, fwd=fwd, fwd_d=fwd_d)

    def greedy_probe(self, Q, starts, layer=0, stream=None):
        """henn_greedy_probe: GreedySearch on one layer from each start.
        Q [nq, d] and starts [nq, S] (int32 layer positions) are CUDA tensors.
        Returns (node int32 [nq, S], dist float32 [nq, S], hops int32 [nq, S])."""
        import torch

        Q = Q.to(torch.float32).contiguous()
        starts = starts.to(torch.int32).contiguous()
        nq, S = starts.shape
        node = torch.empty((nq, S), dtype=torch.int32, device=Q.device)
        dist = torch.empty((nq, S), dtype=torch.float32, device=Q.device)
        hops = torch.empty((nq, S), dtype=torch.int32, device=Q.device)
        _check(load().henn_greedy_probe(self._h, int(layer), _ptr(Q)[0], nq, _ptr(starts)[0], S, _ptr(node)[0],
                                        _ptr(dist)[0], _ptr(hops)[0], _stream(stream)))
        return node, dist, hops

    def search(self, Q, k=10, ef=64, rerank_mult=4, keys=None, out_stride=None, stats=False,
               warps_per_block=0, hash_bits=0, ef_upper=1, descend_all=0, ef_l1=0, stream=None, out=None,
               exact_upper=0, exact_method=EXACT_SORT, time_kernel=False, team_size=0, tile_n=0):
        """Batched query.  Q on the device -> device outputs (torch); Q on the
        host -> host outputs (numpy), copies inside the call.
        k / ef: int or per-query int32 array on the same side as Q.
        exact_upper / exact_method: the lowest upper layer of at most
        exact_upper points gives its exact candidate set, found by a sort in
        the visited table (EXACT_SORT), one batched distance-tile launch with
        a certified rescore (EXACT_TILES) or a scan (EXACT_SCAN).
        out: (ids, dists) to write into instead of new arrays -- CUDA tensors
        for device queries; for host queries numpy arrays (int64 and float32,
        C-contiguous, shape (nq, stride)).  Page-locked host buffers (for
        instance views of pinned tensors) are read and written in place by the
        kernels -- the queries, and the results when both arrays are; pageable
        ones are staged through device memory by copies.
        time_kernel: record the search launches' device time (last_search_ms).
        team_size: warps per query (1, 2 or 4; same results).
        tile_n: columns per tensor-core tile of the TILES exact layer (128 or 256; same results).
        Returns (ids int64 [nq, stride], dists float32 [nq, stride], stats or None)."""
        L = load()
        sp = SearchParams()
        L.henn_search_params_default(C.byref(sp))
        keep = []
        on_dev_q = _is_torch(Q) and Q.is_cuda
        if _is_torch(Q):
            import torch

            Q = Q.to(torch.float32).contiguous()
        else:
            Q = np.ascontiguousarray(Q, dtype=np.float32)
        _check_rows(Q, self.d)
        nq = Q.shape[0]
        kmax = int(k) if np.isscalar(k) else int(np.max(np.asarray(k.cpu() if _is_torch(k) else k)))
        stride = int(out_stride or kmax)
        if np.isscalar(k):
            sp.k_uniform = int(k)
        else:
            p, _, kk = _ptr(k)
            sp.k = p
            keep.append(kk)
        if np.isscalar(ef):
            sp.ef_uniform = int(ef)
        else:
            p, _, kk = _ptr(ef)
            sp.ef = p
            keep.append(kk)
        sp.rerank_mult = int(rerank_mult)
        sp.warps_per_block = int(warps_per_block)
        sp.hash_bits = int(hash_bits)
        sp.ef_upper = int(ef_upper)
        sp.descend_all = int(descend_all)
        sp.ef_l1 = int(ef_l1)
        sp.exact_upper = int(exact_upper)
        sp.exact_method = int(exact_method)
        sp.time_kernel = int(bool(time_kernel))
        sp.team_size = int(team_size)
        sp.tile_n = int(tile_n)
        if keys is not None:
            p, _, kk = _ptr(keys)
            sp.query_keys = p
            keep.append(kk)
        if on_dev_q:
            import torch

            dev = Q.device
            if out is not None:
                ids, dists = out[0], out[1]
            else:
                ids = torch.empty((nq, stride), dtype=torch.int64, device=dev)
                dists = torch.empty((nq, stride), dtype=torch.float32, device=dev)
            st = torch.empty((nq, 4), dtype=torch.int32, device=dev) if stats else None
        else:
            if out is not None:
                ids, dists = out[0], out[1]
                for a_, dt in ((ids, np.int64), (dists, np.float32)):
                    if (not isinstance(a_, np.ndarray) or a_.dtype != dt or a_.shape != (nq, stride)
                            or not a_.flags.c_contiguous or not a_.flags.writeable):
                        raise HennError(1, f"out: host queries need writable C-contiguous numpy arrays of shape "
                                           f"({nq}, {stride}), int64 ids and float32 distances")
            else:
                ids = np.empty((nq, stride), np.int64)
                dists = np.empty((nq, stride), np.float32)
            st = np.empty((nq, 4), np.int32) if stats else None
        if st is not None:
            sp.stats = _ptr(st)[0]
        qp, _, kq = _ptr(Q)
        _check(L.henn_search(self._h, qp, nq, int(on_dev_q), C.byref(sp), _ptr(ids)[0], _ptr(dists)[0], stride,
                             _stream(stream)))
        del keep, kq
        return ids, dists, st

    def last_search_ms(self):
        """(device ms of the search launches, kernel launches) of the last
        search made with time_kernel=True (henn_last_search_ms)."""
        ms = C.c_float()
        n = C.c_int32()
        _check(load().henn_last_search_ms(self._h, C.byref(ms), C.byref(n)))
        return float(ms.value), int(n.value)


def search_host_noalloc(index: "Index", Q, k=10, ef=64, ef_upper=1, out_stride=None, stream=None):
    """henn_search_host_noalloc: host queries and results, no device
    allocation (scratch in the library's fixed 16 MiB device array)."""
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    _check_rows(Q, index.d)
    nq = Q.shape[0]
    stride = int(out_stride or k)
    ids = np.empty((nq, stride), np.int64)
    dd = np.empty((nq, stride), np.float32)
    _check(load().henn_search_host_noalloc(index.handle, C.c_void_p(Q.ctypes.data), nq, int(k), int(ef),
                                           int(ef_upper), C.c_void_p(ids.ctypes.data), C.c_void_p(dd.ctypes.data),
                                           stride, _stream(stream)))
    return ids, dd


class Server:
    """Continuous-batching server over an Index (henn_serve_*).  submit()
    returns a request id, or None when the ring / slots are full (retry
    after polling); poll() returns None while the request runs, else
    (ids int64 [nq, k], dists float32 [nq, k])."""

    def __init__(self, index: "Index", ring_rows=65536, max_requests=1024, max_k=100, max_ef=512, ef_upper=1,
                 descend_all=0, rerank_mult=4, idle_ms=20, ef_l1=0, exact_upper=0):
        L = load()
        p = ServeParams()
        L.henn_serve_params_default(C.byref(p))
        p.ring_rows, p.max_requests, p.max_k, p.max_ef = ring_rows, max_requests, max_k, max_ef
        p.ef_upper, p.descend_all, p.rerank_mult, p.idle_ms = ef_upper, descend_all, rerank_mult, idle_ms
        p.ef_l1, p.exact_upper = ef_l1, exact_upper
        h = C.c_void_p()
        _check(L.henn_serve_create(index.handle, C.byref(p), C.byref(h)))
        self._h = h
        self._index = index  # the index must outlive the server
        self._meta = {}

    def submit(self, Q, k=10, ef=64, keys=None):
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        _check_rows(Q, self._index.d)
        kk = None if keys is None else np.ascontiguousarray(keys, dtype=np.uint64)
        rid = C.c_int64()
        st = load().henn_serve_submit(self._h, C.c_void_p(Q.ctypes.data), Q.shape[0], int(k), int(ef),
                                      None if kk is None else C.c_void_p(kk.ctypes.data), C.byref(rid))
        if st == BUSY:
            return None
        _check(st)
        self._meta[rid.value] = (Q.shape[0], int(k))
        return rid.value

    def poll(self, rid):
        nq, k = self._meta.get(rid, (1, 1))  # unknown ids: the library reports the error
        ids = np.empty((nq, k), np.int64)
        dd = np.empty((nq, k), np.float32)
        done = C.c_int32()
        _check(load().henn_serve_poll(self._h, int(rid), C.byref(done), C.c_void_p(ids.ctypes.data),
                                      C.c_void_p(dd.ctypes.data)))
        if not done.value:
            return None
        self._meta.pop(rid, None)
        return ids, dd

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().henn_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exact_knn(X, Q, k, metric=L2, stream=None):
    """Exact k nearest neighbours on the device (torch CUDA tensors)."""
    import torch

    X = X.to(torch.float32).contiguous()
    Q = Q.to(torch.float32).contiguous()
    ids = torch.empty((Q.shape[0], k), dtype=torch.int64, device=Q.device)
    dd = torch.empty((Q.shape[0], k), dtype=torch.float32, device=Q.device)
    _check(load().henn_exact_knn(_ptr(X)[0], X.shape[0], X.shape[1], _ptr(Q)[0], Q.shape[0], k, metric,
                                 _ptr(ids)[0], _ptr(dd)[0], _stream(stream)))
    return ids, dd


def quantize_rows(X, storage, stream=None):
    """BF16 (uint16 bits) or FP8 E4M3 (uint8 codes + per-row scales) copies."""
    import torch

    X = X.to(torch.float32).contiguous()
    n, d = X.shape
    if storage == BF16:
        out = torch.empty((n, d), dtype=torch.int16, device=X.device)
        scales = None
    else:
        out = torch.empty((n, d), dtype=torch.uint8, device=X.device)
        scales = torch.empty((n,), dtype=torch.float32, device=X.device)
    _check(load().henn_quantize_rows(_ptr(X)[0], n, d, storage, _ptr(out)[0],
                                     _ptr(scales)[0] if scales is not None else None, _stream(stream)))
    return out, scales
