"""henn_search_host_noalloc: the search for callers that cannot allocate
device memory (their device memory belongs to another allocator, or they
must not allocate while running).  Its scratch is the library's fixed
device array, so its results must equal those of henn_search with host
buffers, call after call, for every storage form, metric and beam width
the entry point accepts.  Collected last so that a failure here comes
after every other test has run."""
from __future__ import annotations

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_17368_gb300 as H  # noqa: E402
from paper_2505_17368_gb300 import binding  # noqa: E402

_INDEXES = {}


def _index(storage, metric):
    key = (storage, metric)
    if key not in _INDEXES:
        if metric == H.L2:
            X, Q, _ = synth.workload("uniform-10k-d32")
        else:
            X, _ = synth.gaussian_mixture(10000, 48, 40, seed=0, normalise=True)
            Q, _ = synth.gaussian_mixture(1000, 48, 40, seed=1, normalise=True)
        _INDEXES[key] = (H.Index(X, seed=0, storage=storage, metric=metric), Q)
    return _INDEXES[key]


@pytest.fixture(scope="module")
def index_and_queries():
    return _index(H.F32, H.L2)


def test_no_alloc_equals_search_two_calls_in_a_row(index_and_queries):
    idx, Q = index_and_queries
    ref_ids, ref_d, _ = idx.search(Q, k=10, ef=64)
    for _ in range(2):
        ids, dd = binding.search_host_noalloc(idx, Q, k=10, ef=64)
        assert np.array_equal(ids, ref_ids)
        assert np.array_equal(dd, ref_d)
    # a different batch right after: the shared array keeps the previous
    # call's contents, which must not leak into this one
    ref2, refd2, _ = idx.search(Q[:137], k=5, ef=40, ef_upper=8, out_stride=7)
    ids2, dd2 = binding.search_host_noalloc(idx, Q[:137], k=5, ef=40, ef_upper=8, out_stride=7)
    assert np.array_equal(ids2, ref2) and np.array_equal(dd2, refd2)


@pytest.mark.parametrize("storage", [H.F32, H.BF16, H.FP8E4M3])
@pytest.mark.parametrize("metric", [H.L2, H.ANGULAR])
@pytest.mark.parametrize("ef", [64, 128, 4096])
def test_no_alloc_equals_search_every_form(storage, metric, ef):
    """Same launch shape and results as henn_search (default rerank of the
    best 4k for BF16 / FP8), two calls in a row, up to the widest beam."""
    idx, Q = _index(storage, metric)
    Qs = Q[:100] if ef > 1000 else Q[:400]
    ref_ids, ref_d, _ = idx.search(Qs, k=10, ef=ef, ef_upper=4, rerank_mult=4)
    for _ in range(2):
        ids, dd = binding.search_host_noalloc(idx, Qs, k=10, ef=ef, ef_upper=4)
        assert np.array_equal(ids, ref_ids)
        assert np.array_equal(dd, ref_d)


def test_no_alloc_rejects_batches_beyond_the_scratch(index_and_queries):
    idx, Q = index_and_queries
    big = np.repeat(Q, 80, axis=0)  # 80,000 queries x (128 + 120) bytes > 16 MiB
    with pytest.raises(H.HennError) as e:
        binding.search_host_noalloc(idx, big, k=10, ef=64)
    assert e.value.status == 1 and "scratch" in str(e.value)
    # rows of the wrong width are refused before the library reads them
    with pytest.raises(H.HennError) as e:
        binding.search_host_noalloc(idx, Q[:, :16], k=10, ef=64)
    assert e.value.status == 1
    # still usable afterwards
    ids, _ = binding.search_host_noalloc(idx, Q[:10], k=10, ef=64)
    ref, _, _ = idx.search(Q[:10], k=10, ef=64)
    assert np.array_equal(ids, ref)
