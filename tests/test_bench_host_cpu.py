"""Host logic of the benchmark on CPU: the CIGAR capacity it allocates holds every accepted pair's runs, the plain
form's read-length groups cover the pairs exactly once, and the DRAM-traffic record is used only while the
kernel source still has the hash it was captured at."""
import hashlib
import json
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import gen  # noqa: E402
import oracle  # noqa: E402


@pytest.mark.parametrize("name,count", [("wfa_uneven", 400), ("edit_nw_100bp", 2_000), ("gotoh_250bp", 1_000)])
def test_runs_capacity_holds_every_accepted_alignment(oracle_lib, gen_lib, name, count):
    w = bench.WORKLOADS[name]
    algo = bench.ALGO_OF[name]
    p = gen.generate(w, count)
    cap = bench.runs_capacity(w, p, algo)
    me = gen.per_pair_max_edits(w, p)
    unit = algo in ("edit", "genasm")
    pen = oracle.UNIT if unit else w.penalties
    lim = np.array([oracle.limit_for(w.penalties, int(k), unit=unit) for k in me], np.int64)
    band = w.band if algo == "gotoh" else -1
    s, f, off, cig, lens = oracle.align_batch(p, pen, lim, band=band)
    ok = f == 0
    assert ok.any()
    assert (lens[ok] <= cap[ok]).all()


def test_runs_capacity_holds_genasm_runs(oracle_lib, gen_lib):
    w = gen.GENASM[(150, 5)]
    p = gen.generate(w, 2_000)
    cap = bench.runs_capacity(w, p, "genasm")
    lim = np.full(len(p), w.max_edits, np.int64)
    s, f, off, cig, lens = oracle.genasm_batch(p, lim)
    ok = f == 0
    assert ok.any() and (lens[ok] <= cap[ok]).all()


def test_length_groups_cover_every_pair_once(gen_lib):
    p = gen.generate(gen.WFA_UNEVEN, 5_000)
    groups = bench.length_groups(p)
    allidx = np.sort(np.concatenate(groups))
    assert np.array_equal(allidx, np.arange(len(p)))
    for g in groups[:-1]:
        assert p.read_len[g].max() < 1001


def test_traffic_record_follows_the_source_hash(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2208_01243_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "k.cu"
    hdr = src_dir / "h.cuh"
    src.write_bytes(b"__global__ void k() {}\n")
    hdr.write_bytes(b"// shared\n")
    sha = hashlib.sha256(src.read_bytes() + hdr.read_bytes()).hexdigest()[:16]
    rec = {"k:w": {"sources": ["k.cu", "h.cuh"], "sources_sha": sha, "dram_bytes_per_launch": 123, "how": "test"}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("k", "w")["dram_bytes_per_launch"] == 123
    assert bench.traffic_record("k", "other") is None
    hdr.write_bytes(b"// shared, changed\n")          # a change to the shared header voids the record too
    assert bench.traffic_record("k", "w") is None
    hdr.write_bytes(b"// shared\n")
    assert bench.traffic_record("k", "w")["dram_bytes_per_launch"] == 123
    src.write_bytes(b"__global__ void k() { /* changed */ }\n")
    assert bench.traffic_record("k", "w") is None
