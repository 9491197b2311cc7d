"""Failure detection without a GPU fault: the tensor-core tile pipeline's
bounded waits.  The host tells the pipeline's TMA producer to issue nothing
(HENN_TILE_HOLD_LOADS, a delivery that never comes) and shortens the wait
bound (HENN_TILE_SPIN_LIMIT); the MMA and epilogue warps' waits then run
out with no copy or MMA in flight, the blocks free their tensor memory and
return, and henn_build reports HENN_ERR_TIMEOUT.  The same process then
builds and searches normally: the context stays usable.  Run in a child
process so the environment switches cannot reach other tests."""
from __future__ import annotations

import os
import subprocess
import sys
import time

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_2505_17368_gb300 as H
import synth
X = synth.uniform_cube(3000, 32, seed=3)
os.environ["HENN_TILE_HOLD_LOADS"] = "1"
os.environ["HENN_TILE_SPIN_LIMIT"] = "256"
t0 = time.time()
try:
    H.Index(X, seed=0, tiles=H.TILES_TCGEN05)
    print("NO_ERROR")
except H.HennError as e:
    print("STATUS", e.status, "SECONDS", round(time.time() - t0, 3))
del os.environ["HENN_TILE_HOLD_LOADS"]
del os.environ["HENN_TILE_SPIN_LIMIT"]
idx = H.Index(X, seed=0, tiles=H.TILES_TCGEN05)
ids, _, _ = idx.search(X[:5], k=1, ef=16)
print("AFTER", ids[:, 0].tolist())
"""


def test_tile_pipeline_wait_runs_out_and_reports_timeout():
    t0 = time.time()
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = r.stdout
    assert "STATUS 5 " in out, out  # HENN_ERR_TIMEOUT
    assert "AFTER [0, 1, 2, 3, 4]" in out, out
    assert time.time() - t0 < 300
