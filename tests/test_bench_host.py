"""Host logic of bench.py (no GPU): the sweep's beam entries and the lookup of
the search kernel's DRAM bytes in the committed ncu summary."""
from __future__ import annotations

import hashlib
import os

import bench


def test_sweep_entries_are_well_formed():
    for entry in bench.UPPER_SWEEP:
        assert len(entry) in (5, 6), entry
        efu, da, l1, xu, xm = entry[:5]
        assert efu >= 0 and da in (0, 1) and l1 >= 0 and xm in (0, 1, 2)
        assert isinstance(xu, int) or (isinstance(xu, str) and xu[0] == "L" and xu[1:].isdigit())
        if xm != 0 and da:
            assert efu <= 32  # the tile and scan methods keep at most 32 seeds
        if len(entry) == 6:
            assert entry[5] >= 1
    assert bench.EF_SWEEP == sorted(bench.EF_SWEEP)


def _tree(tmp_path, src, lines):
    csrc = tmp_path / "paper_2505_17368_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "search.cu").write_bytes(src)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "search_bf16_mixture-1m-d128.md").write_text("# summary\n\n" + "".join(f"- {l}\n" for l in lines))


def test_profile_traffic_lookup(tmp_path, monkeypatch):
    src = b"// kernel source\n"
    sha = hashlib.sha256(src).hexdigest()[:16]
    _tree(tmp_path, src, [
        f"search.cu sha256[:16]: {sha}",
        "dram bytes per launch [ef=48 ef_upper=8 descend_all=1 ef_l1=0 exact_upper=3677 exact_method=1]: 111",
        "dram bytes per launch [ef=48 ef_upper=8 descend_all=1 ef_l1=0 exact_upper=3677 exact_method=1 "
        "rerank_mult=2]: 222",
    ])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    beam = (48, 8, 1, 0, 3677, 1)
    assert bench._profile_traffic(beam) == 111.0
    assert bench._profile_traffic(beam, 2) == 222.0
    assert bench._profile_traffic(beam, 3) is None
    assert bench._profile_traffic((44, 16, 1, 0, 3677, 1)) is None
    # a summary taken on another kernel source is not used
    (tmp_path / "paper_2505_17368_gb300" / "csrc" / "search.cu").write_bytes(src + b"// changed\n")
    assert bench._profile_traffic(beam) is None


def test_profile_traffic_without_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert not os.path.exists(tmp_path / "profiles")
    assert bench._profile_traffic((48, 8, 1, 0, 3677, 1)) is None
