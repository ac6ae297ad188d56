"""GenASM on the GPU vs the oracle, element by element (scores, flags, CIGAR runs).

The kernel computes bitap status vectors level by level and traces back from
them; the oracle fills the suffix edit-distance table of each window and
traces back from that.  Sizes here span many warps, ragged tails, one to
hundreds of windows per pair, windows of 1 to 64 bases, and every edge of the
window rule (free and ending sides, the last window).
"""
import numpy as np
import pytest

import gen
import oracle
from devutil import assert_same, device_results
from oracle.cigar import cost, decode, reconstruct_target

pytestmark = pytest.mark.gpu

UNIT = oracle.UNIT


@pytest.fixture(scope="module")
def aligner():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim
    a = aim.Aligner(0, 4 << 30)
    yield a
    a.close()


@pytest.fixture
def window(aligner):
    """Set the GenASM window on the shared context for one test, then restore the defaults."""
    import paper_2208_01243_gb300 as aim

    def set_(W, O):
        aim.aim_set_genasm_window(aligner.ctx, W, O)
    yield set_
    aim.aim_set_genasm_window(aligner.ctx, oracle.GENASM_W, oracle.GENASM_O)


def oracle_genasm(p, k, W=oracle.GENASM_W, O=oracle.GENASM_O, per_pair=None):
    lim = (per_pair.astype(np.int64) if per_pair is not None
           else np.full(len(p), (1 << 62) if k < 0 else k, np.int64))
    s, f, off, cig, lens = oracle.genasm_batch(p, lim, W=W, O=O)
    return s, f, [cig[off[i]:off[i] + lens[i]].astype(np.uint32) for i in range(len(p))]


@pytest.mark.parametrize("key,count", [((100, 1), 20_011), ((100, 5), 20_011), ((150, 1), 20_011),
                                       ((150, 5), 20_011), ((250, 1), 6_007), ((250, 5), 6_007),
                                       ((1000, 1), 1_003), ((1000, 5), 1_003)])
def test_paper_shapes(aligner, oracle_lib, gen_lib, key, count):
    w = gen.GENASM[key]
    p = gen.generate(w, count)
    dev = device_results(p, "genasm", UNIT, w.max_edits, aligner=aligner)
    assert_same(dev, oracle_genasm(p, w.max_edits), what=f"genasm {key}")


def test_packed_path_and_unrelated_pairs(aligner, oracle_lib, gen_lib):
    w = gen.Workload("genasm_150bp_5pct_unrel30", 81, 8_191, 150, 150, 0.05, 0.05, 0.3, "genasm", UNIT, 8)
    p = gen.generate(w)
    orc = oracle_genasm(p, 8)
    for path in ("ascii", "packed"):
        dev = device_results(p, "genasm", UNIT, 8, path=path, aligner=aligner)
        assert_same(dev, orc, what=f"genasm unrelated {path}")
    rej = (dev[1] & oracle.F_REJECTED) > 0
    assert rej.sum() > 0.25 * len(p) and (dev[0][rej] == -1).all()


def test_per_pair_thresholds_uneven_lengths(aligner, oracle_lib, gen_lib):
    w = gen.Workload("genasm_uneven", 82, 5_003, 30, 3000, 0.0, 0.12, 0.05, "genasm", UNIT, None,
                     max_edits_frac=0.08)
    p = gen.generate(w)
    pp = gen.per_pair_max_edits(w, p)
    bound = int(pp.max())
    dev = device_results(p, "genasm", UNIT, bound, per_pair=pp, aligner=aligner)
    assert_same(dev, oracle_genasm(p, bound, per_pair=pp), what="genasm per-pair thresholds")


@pytest.mark.parametrize("W,O", [(1, 0), (2, 1), (3, 0), (4, 1), (7, 3), (16, 4), (31, 10), (32, 8), (33, 32),
                                 (63, 0), (64, 63)])
def test_window_sizes(aligner, window, oracle_lib, gen_lib, W, O):
    w = gen.Workload("genasm_windows", 83, 3_001, 0, 200, 0.0, 0.25, 0.1, "genasm", UNIT, None)
    p = gen.generate(w)
    window(W, O)
    for k in (-1, 12):
        dev = device_results(p, "genasm", UNIT, k, aligner=aligner)
        assert_same(dev, oracle_genasm(p, k, W, O), what=f"genasm W={W} O={O} k={k}")


def test_edge_lengths(aligner, oracle_lib, gen_lib):
    """Lengths at and around word and window boundaries, empty sides, identical and all-mismatch pairs."""
    rnd = np.random.default_rng(5)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    reads, targets = [], []
    for L in (0, 1, 2, 31, 32, 33, 63, 64, 65, 96, 127, 128, 129, 200):
        for L2 in (0, 1, L, L + 1, max(L - 1, 0), 64, 65, 130):
            r = rnd.choice(acgt, L).tobytes()
            reads.append(r)
            targets.append(r[:L2] if L2 <= L else r + rnd.choice(acgt, L2 - L).tobytes())
        reads.append(b"A" * L); targets.append(b"C" * L)
        reads.append(b"A" * L); targets.append(b"C" * (L // 2))
        s = rnd.choice(acgt, L).tobytes()
        reads.append(s); targets.append(s)
    p = gen.from_strings(reads, targets)
    for k in (-1, 0, 5, 64):
        dev = device_results(p, "genasm", UNIT, k, aligner=aligner)
        assert_same(dev, oracle_genasm(p, k), what=f"genasm edges k={k}")


def test_long_reads_many_windows(aligner, oracle_lib, gen_lib):
    w = gen.Workload("genasm_long", 84, 61, 5000, 12000, 0.01, 0.08, 0.0, "genasm", UNIT, None)
    p = gen.generate(w)
    dev = device_results(p, "genasm", UNIT, -1, aligner=aligner)
    assert_same(dev, oracle_genasm(p, -1), what="genasm long reads")
    for i in range(0, len(p), 10):
        assert dev[0][i] >= oracle.levenshtein(p.read(i), p.target(i))


def test_max_score_and_ragged_counts(aligner, oracle_lib, gen_lib):
    import paper_2208_01243_gb300 as aim
    w = gen.GENASM[(150, 5)]
    for count in (1, 31, 33, 129):
        p = gen.generate(w, count)
        dev = device_results(p, "genasm", UNIT, 100, max_score=5, aligner=aligner)   # max_score overrides
        assert_same(dev, oracle_genasm(p, 5), what=f"genasm max_score count={count}")
    with pytest.raises(aim.AimError):
        device_results(gen.generate(w, 4), "genasm", UNIT, 8, band=10, aligner=aligner)


def test_cigar_overflow_keeps_score(aligner, oracle_lib, gen_lib):
    w = gen.GENASM[(150, 5)]
    p = gen.generate(w, 2_000)
    s, f, runs = oracle_genasm(p, -1)
    cap = np.full(len(p), 5, np.int64)
    dev = device_results(p, "genasm", UNIT, -1, cigar_cap=cap, aligner=aligner)
    n_runs = np.array([len(r) for r in runs])
    assert (dev[0] == s).all()
    assert (dev[3] == n_runs).all()
    over = n_runs > 5
    assert over.any()
    assert ((dev[1] & oracle.F_CIGAR_OVERFLOW) > 0).tolist() == over.tolist()
    for i in np.flatnonzero(~over):
        assert np.array_equal(dev[2][i], runs[i])


def test_bad_inputs(aligner, oracle_lib, gen_lib):
    p = gen.from_strings([b"ACGT", b"ACNT", b"ACGTACGT", b"ACG"], [b"ACGT", b"ACGT", b"ACGTACGT", b"ACGA"])
    dev = device_results(p, "genasm", UNIT, 3, max_length=4, aligner=aligner)
    assert dev[1].tolist() == [0, oracle.F_BAD_PAIR, oracle.F_BAD_PAIR, 0]
    assert dev[0].tolist() == [0, -1, -1, 1]
    pp = np.array([1, 2, 9, 3], np.int32)   # 9 exceeds the stated bound 3
    dev = device_results(p, "genasm", UNIT, 3, per_pair=pp, aligner=aligner)
    assert dev[1].tolist() == [0, oracle.F_BAD_PAIR, oracle.F_BAD_PAIR, 0]


def test_full_size_150bp_sampled(aligner, oracle_lib, gen_lib):
    """All 1M pairs of the 150 bp, 5 % workload on the device; a seeded sample against the oracle; properties
    of every pair."""
    import paper_2208_01243_gb300 as aim
    w = gen.GENASM[(150, 5)]
    p = gen.generate(w)
    aim.aim_stats_reset(aligner.ctx)
    dev = device_results(p, "genasm", UNIT, w.max_edits, aligner=aligner)
    st = aim.aim_stats_read(aligner.ctx)
    assert st["pairs"] == len(p) and st["bitap_words"] > 0
    rng = np.random.default_rng(17)
    idx = np.sort(rng.choice(len(p), 3000, replace=False))
    sub = gen.generate(w, index=idx)
    orc = oracle_genasm(sub, w.max_edits)
    assert_same(dev, orc, idx=list(idx), what="genasm 1M sample")
    ok = dev[1] == 0
    assert ok.mean() > 0.99 and (dev[0][ok] <= w.max_edits).all()
    for i in idx[:300]:
        ops = decode(dev[2][i])
        assert cost(ops, p.read(i), p.target(i), UNIT) == dev[0][i]
        assert reconstruct_target(ops, p.read(i)) is not None


def test_small_workspace_still_exact(oracle_lib, gen_lib):
    import paper_2208_01243_gb300 as aim
    w = gen.GENASM[(250, 5)]
    p = gen.generate(w, 3_001)
    small = aim.Aligner(0, 8 << 20)       # a few warps of scratch only
    try:
        dev = device_results(p, "genasm", UNIT, w.max_edits, aligner=small)
        assert_same(dev, oracle_genasm(p, w.max_edits), what="genasm small workspace")
    finally:
        small.close()
    tiny = aim.Aligner(0, 64 << 10)       # not even one warp's scratch
    try:
        with pytest.raises(aim.AimError):
            device_results(gen.generate(w, 4), "genasm", UNIT, w.max_edits, aligner=tiny)
    finally:
        tiny.close()
