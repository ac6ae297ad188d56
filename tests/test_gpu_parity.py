"""CUDA path vs the oracle, element by element (scores, flags, CIGAR runs).

Sizes the oracle finishes in seconds span many warps and a ragged tail
(counts not a multiple of the 8 warps of a block or of the grid); the full
sizes of the large workloads are run on the device in full and checked on a
seeded sample against the oracle plus whole-batch properties.
"""
import numpy as np
import pytest

import gen
import oracle
from devutil import assert_same, device_results, limits, oracle_results
from oracle.cigar import cost, decode

pytestmark = pytest.mark.gpu

AFF = (0, 4, 6, 2)


@pytest.fixture(scope="module")
def aligner():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim
    a = aim.Aligner(0, 4 << 30)
    yield a
    a.close()


@pytest.mark.parametrize("path", ["ascii", "packed"])
def test_edit_nw_100bp_all_pairs(aligner, oracle_lib, gen_lib, path):
    w = gen.EDIT_NW_100BP
    p = gen.generate(w)                       # all 10,000 pairs
    orc = oracle_results(p, oracle.UNIT, limits(w, p))
    dev = device_results(p, "edit", oracle.UNIT, 10, path=path, aligner=aligner)
    assert_same(dev, orc, what=f"edit nw {path}")
    # the textbook Levenshtein agrees with the scores on a sample
    for i in range(0, len(p), 997):
        assert dev[0][i] == oracle.levenshtein(p.read(i), p.target(i))


def test_wfa_150bp_parity_small(aligner, oracle_lib, gen_lib):
    w = gen.WFA_150BP
    p = gen.generate(w, 20_011)
    orc = oracle_results(p, AFF, limits(w, p))
    dev = device_results(p, "wfa", AFF, 6, aligner=aligner)
    assert_same(dev, orc, what="wfa 150bp")
    rej = (dev[1] & oracle.F_REJECTED) > 0
    assert rej.sum() > 0 and (rej <= p.unrelated.astype(bool)).all()   # only unrelated pairs are rejected


@pytest.mark.parametrize("algo", ["gotoh", "wfa"])
def test_gotoh_wfa_250bp_band25_parity_small(aligner, oracle_lib, gen_lib, algo):
    w = gen.GOTOH_WFA_250BP
    p = gen.generate(w, 3_001)
    orc = oracle_results(p, AFF, limits(w, p), band=25)
    dev = device_results(p, algo, AFF, 25, band=25, aligner=aligner)
    assert_same(dev, orc, what=f"{algo} band 25")


@pytest.mark.parametrize("lanes", [4, 32])
def test_wfa_deferred_tracebacks_any_workspace(oracle_lib, gen_lib, lanes):
    """Groups defer their tracebacks as far as their share of the scratch allows: one pair per flush when the
    arena holds one pair's planned need, several when it holds more, up to G, and a last flush when the queue is
    drained.  30k pairs keep every warp busy with several pairs.  Results never depend on it."""
    import paper_2208_01243_gb300 as aim
    w = gen.WFA_150BP
    p = gen.generate(w, 30_011)
    orc = oracle_results(p, AFF, limits(w, p))
    for ws in (16 << 20, 96 << 20, 2 << 30):
        al = aim.Aligner(0, ws)
        try:
            aim.aim_set_wfa_group(al.ctx, lanes)
            dev = device_results(p, "wfa", AFF, w.max_edits, aligner=al)
        finally:
            al.close()
        assert_same(dev, orc, what=f"wfa lanes={lanes} workspace={ws >> 20} MiB")


@pytest.mark.parametrize("algo", ["gotoh", "edit"])
def test_dp_deferred_tracebacks_any_workspace(oracle_lib, gen_lib, algo):
    """The banded DP keeps up to 32 finished pairs per warp for side-by-side tracebacks, as many slots as the
    scratch spread over the warps allows: 1 with 40 MiB, a few with 320 MiB (flushes whenever they fill), many
    with 4 GiB.  Results never depend on it."""
    w = gen.GOTOH_WFA_250BP
    p = gen.generate(w, 20_003)
    pen = AFF if algo == "gotoh" else oracle.UNIT
    lim = np.array([oracle.limit_for(pen, 25, unit=algo == "edit")] * len(p), np.int64)
    orc = oracle_results(p, pen, lim, band=25)
    for ws in (40 << 20, 320 << 20, 4 << 30):
        dev = device_results(p, algo, pen, 25, band=25, workspace=ws)
        assert_same(dev, orc, what=f"{algo} band 25 workspace={ws >> 20} MiB")


def test_wfa_uneven_parity_sample(aligner, oracle_lib, gen_lib):
    w = gen.WFA_UNEVEN
    p = gen.generate(w, 1_500)
    me = gen.per_pair_max_edits(w, p)
    orc = oracle_results(p, AFF, limits(w, p))
    dev = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, aligner=aligner)
    assert_same(dev, orc, what="wfa uneven")


def test_unbanded_gotoh_equals_wfa(aligner, gen_lib):
    """Gotoh with the band derived from the limit (exact) == WFA, CIGAR included."""
    p = gen.generate(gen.WFA_150BP, 10_007)
    a = device_results(p, "gotoh", AFF, 6, aligner=aligner)
    b = device_results(p, "wfa", AFF, 6, aligner=aligner)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert all(np.array_equal(x, y) for x, y in zip(a[2], b[2]))


def test_wfa_150bp_full_size(aligner, oracle_lib, gen_lib):
    """All 1,000,000 pairs on the device; a seeded sample against the oracle; properties on the rest."""
    w = gen.WFA_150BP
    p = gen.generate(w)
    dev = device_results(p, "wfa", AFF, 6, aligner=aligner)
    s, f = dev[0], dev[1]
    rej = (f & oracle.F_REJECTED) > 0
    assert not (f & ~np.uint8(oracle.F_REJECTED)).any()
    related = ~p.unrelated.astype(bool)
    assert not rej[related].any()                      # <= 6 edits never exceed 6 * 8
    bound = gen.script_cost_bound(p, 4, 6, 2)
    assert (s[related] <= bound[related]).all() and (s[related] >= 0).all()
    idx = np.random.default_rng(2).choice(len(p), 3000, replace=False)
    sub = gen.generate(w, index=idx)
    orc = oracle_results(sub, AFF, limits(w, sub))
    assert_same(dev, orc, idx=idx, what="wfa 150bp full-size sample")
    for i in idx[:500]:
        if not rej[i]:
            assert cost(decode(dev[2][i]), p.read(i), p.target(i), AFF) == s[i]


def test_gotoh_wfa_250bp_full_size_cross_check(aligner, oracle_lib, gen_lib):
    """1,000,000 pairs: banded Gotoh and banded WFA agree bit for bit; a sample matches the oracle."""
    w = gen.GOTOH_WFA_250BP
    p = gen.generate(w)
    a = device_results(p, "gotoh", AFF, 25, band=25, aligner=aligner)
    b = device_results(p, "wfa", AFF, 25, band=25, aligner=aligner)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])
    assert all(np.array_equal(x, y) for x, y in zip(a[2], b[2]))
    idx = np.random.default_rng(3).choice(len(p), 1000, replace=False)
    sub = gen.generate(w, index=idx)
    assert_same(a, oracle_results(sub, AFF, limits(w, sub), band=25), idx=idx, what="gotoh 250bp sample")


# ---------------- edge cases ----------------

EDGE_READS = ["", "", "A", "ACGT", "A" * 31, "C" * 32, "G" * 33, "ACGT" * 16, "ACGT" * 16 + "A", "T" * 65,
              "AAAA", "GATTACA", "ACGTACGT", "ACGTTGCA", "A" * 40]
EDGE_TARGS = ["", "ACG", "", "ACGT", "A" * 32, "C" * 31, "G" * 33, "ACGT" * 16 + "A", "ACGT" * 16, "T" * 64,
              "CCCC", "GCATTAC", "ACTTACGGT", "ACGTTGCA", "C" * 40]


@pytest.mark.parametrize("algo,pen", [("edit", oracle.UNIT), ("gotoh", AFF), ("wfa", AFF), ("wfa", (0, 3, 4, 1)),
                                      ("gotoh", (0, 2, 1, 1))])
def test_edge_cases(aligner, oracle_lib, algo, pen):
    p = gen.from_strings(EDGE_READS, EDGE_TARGS)
    for max_edits in (-1, 0, 3):
        if algo != "wfa" and max_edits < 0:
            continue          # the DP needs a band; unbounded below is covered by the WFA
        unit = algo == "edit"
        lim = np.full(len(p), oracle.limit_for(pen, max_edits, unit=unit), np.int64)
        orc = oracle_results(p, pen, lim)
        dev = device_results(p, algo, pen, max_edits, aligner=aligner)
        assert_same(dev, orc, what=f"edges {algo} {pen} max_edits={max_edits}")


def test_max_score_overrides_and_bands(aligner, oracle_lib, gen_lib):
    p = gen.generate(gen.WFA_150BP, 500)
    for band in (-1, 3, 10):
        for algo in ("wfa", "gotoh"):
            if algo == "gotoh" and band < 0:
                continue
            lim = np.full(len(p), 30, np.int64)
            orc = oracle_results(p, AFF, lim, band=band)
            dev = device_results(p, algo, AFF, 6, band=band, max_score=30, aligner=aligner)
            assert_same(dev, orc, what=f"{algo} band {band} max_score 30")


def test_bad_inputs_flagged(aligner, oracle_lib):
    p = gen.from_strings(["ACGT", "ACNT", "ACGT", "A" * 50], ["ACGT", "ACGT", "ACGX", "A" * 50])
    dev = device_results(p, "wfa", AFF, 2, max_length=40, aligner=aligner)
    assert list(dev[1]) == [0, 4, 4, 4] and list(dev[0]) == [0, -1, -1, -1]
    # per-pair threshold above the stated bound
    dev = device_results(p, "wfa", AFF, 2, per_pair=np.array([1, 1, 1, 3], np.int32), aligner=aligner)
    assert dev[1][3] == 4


def test_cigar_overflow_reports_length(aligner, oracle_lib):
    p = gen.from_strings(["ACGTACGT", "GATTACA"], ["ACTTACGGT", "GCATTAC"])
    dev = device_results(p, "wfa", AFF, -1, cigar_cap=np.array([2, 20]), aligner=aligner)
    assert dev[1][0] == oracle.F_CIGAR_OVERFLOW and dev[3][0] == 5 and dev[0][0] == 12
    assert dev[1][1] == 0 and decode(dev[2][1]) == "MDMMMMMI"


def test_device_packer_matches_layout(aligner):
    import torch
    import paper_2208_01243_gb300 as aim
    from oracle import pack
    rng = np.random.default_rng(5)
    seqs = [rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(L)).tobytes()
            for L in [0, 1, 31, 32, 33, 63, 64, 65, 100, 1000, 5]]
    seqs.append(b"ACGTN" + b"A" * 40)
    lens = np.array([len(s) for s in seqs], np.uint32)
    co = np.zeros(len(seqs), np.int64); co[1:] = np.cumsum(lens[:-1])
    wo = np.zeros(len(seqs), np.int64); wo[1:] = np.cumsum((lens[:-1].astype(np.int64) + 31) // 32)
    total = int(wo[-1] + (int(lens[-1]) + 31) // 32)
    ascii_, l_, co_, wo_ = aim.upload(np.frombuffer(b"".join(seqs), np.uint8), lens, co, wo)
    packed = torch.full((total,), -1, dtype=torch.int64, device=ascii_.device)
    bad = torch.zeros(len(seqs), dtype=torch.uint8, device=ascii_.device)
    aim.aim_pack_2bit(aligner.ctx, ascii_, co_, l_, packed, wo_, bad)
    torch.cuda.synchronize()
    got = packed.cpu().numpy().view(np.uint64)
    for i, s in enumerate(seqs[:-1]):
        want = np.array(pack.pack_one(s), np.uint64)
        assert np.array_equal(got[wo[i]:wo[i] + len(want)], want), i
    assert list(bad.cpu().numpy()) == [0] * (len(seqs) - 1) + [1]


@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_ascii_path_odd_buffer_addresses_and_bad_bytes(aligner, oracle_lib, shift):
    """The fixed-slot packer behind the ASCII entry point: input buffers starting at any byte address, lengths
    across partial 4-byte groups and words, and a non-ACGT byte at every position class flags the pair."""
    import torch
    import paper_2208_01243_gb300 as aim
    rng = np.random.default_rng(40 + shift)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    reads, targets, bad = [], [], []
    for L in list(range(0, 70)) + [95, 96, 97, 127, 128, 129, 200]:
        r = bytearray(rng.choice(acgt, L).tobytes())
        t = bytearray(r)
        if L and rng.random() < 0.5:
            t[int(rng.integers(L))] = int(rng.choice(acgt))
        b = False
        if L and L % 5 == 0:   # a bad byte in the read or the target, anywhere
            which = r if L % 10 == 0 else t
            which[int(rng.integers(L))] = int(rng.choice(np.frombuffer(b"Nacgt.", np.uint8)))
            b = True
        reads.append(bytes(r)); targets.append(bytes(t)); bad.append(b)
    p = gen.from_strings(reads, targets)
    n = len(p)
    dev = torch.device("cuda", 0)

    def shifted(a):
        buf = torch.zeros(len(a) + shift + 8, dtype=torch.uint8, device=dev)
        buf[shift:shift + len(a)] = torch.from_numpy(a).to(dev)
        return buf[shift:]                      # a view whose data pointer is `shift` bytes past an aligned one
    rd, td = shifted(p.reads), shifted(p.targets)
    rl, tl, ro, to = aim.upload(p.read_len, p.target_len, p.read_off, p.target_off)
    cap = (p.read_len.astype(np.int64) + p.target_len.astype(np.int64) + 1)
    off = np.zeros(n + 1, np.int64); off[1:] = np.cumsum(cap)
    coff = aim.upload(off)[0]
    scores = torch.full((n,), -7, dtype=torch.int32, device=dev)
    flags = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    lens = torch.zeros(n, dtype=torch.int32, device=dev)
    cig = torch.zeros(int(off[-1]), dtype=torch.int32, device=dev)
    aim.aim_align_batch_ascii(aligner.ctx, rd, td, ro, to, rl, tl, 200, "edit", aim.penalties(1, 0, 1), 100, None,
                              scores, cig, coff, lens, flags)
    torch.cuda.synchronize()
    s_, f_ = scores.cpu().numpy(), flags.cpu().numpy()
    cg = cig.cpu().numpy().view(np.uint32); ln = lens.cpu().numpy()
    for i in range(n):
        if bad[i]:
            assert (s_[i], f_[i]) == (-1, oracle.F_BAD_PAIR), i
            continue
        sc, fl, runs = oracle.align(p.read(i), p.target(i), oracle.UNIT)
        assert (s_[i], f_[i]) == (sc, fl), i
        assert list(cg[off[i]:off[i] + ln[i]]) == runs, i


def test_packer_flags_every_non_acgt_byte(aligner, oracle_lib):
    """Every byte value other than A, C, G and T (lowercase letters, N, NUL, 0xff ...) flags its pair, at any
    position of a word and of a 4-byte group; the pairs without one align as the oracle does."""
    rng = np.random.default_rng(77)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    reads, targets, bad = [], [], []
    for v in range(256):
        if v in acgt:
            continue
        for planted in (True, False):
            L = int(rng.integers(1, 80))
            r = bytearray(rng.choice(acgt, L).tobytes())
            t = bytearray(r)
            t[int(rng.integers(L))] = int(rng.choice(acgt))
            if planted:
                (r if v % 2 else t)[int(rng.integers(L))] = v
            reads.append(bytes(r)); targets.append(bytes(t)); bad.append(planted)
    p = gen.from_strings(reads, targets)
    s, f, runs, _ = device_results(p, "edit", oracle.UNIT, 80, aligner=aligner)
    for i in range(len(p)):
        if bad[i]:
            assert (s[i], f[i]) == (-1, oracle.F_BAD_PAIR), i
        else:
            sc, fl, rr = oracle.align(p.read(i), p.target(i), oracle.UNIT)
            assert (s[i], f[i], list(runs[i])) == (sc, fl, list(rr)), i


def test_dp_huge_costs_keep_the_value_cap(aligner, oracle_lib):
    """Costs of 2^20 over reads of up to 1,000 bp could take DP values past int32 without the cap at infinity, so
    the host picks the capped kernel instance there; results match the oracle."""
    rng = np.random.default_rng(91)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    big = 1 << 20
    pen = (0, big, big, big)
    reads, targets = [], []
    for _ in range(64):
        L = int(rng.integers(900, 1001))
        r = rng.choice(acgt, L)
        t = r.copy()
        for _ in range(int(rng.integers(0, 4))):   # up to three substitutions
            j = int(rng.integers(L))
            t[j] = acgt[(int(np.flatnonzero(acgt == t[j])[0]) + 1) % 4]
        reads.append(r.tobytes()); targets.append(t.tobytes())
    p = gen.from_strings(reads, targets)
    s, f, runs, _ = device_results(p, "gotoh", pen, 3, aligner=aligner)
    for i in range(len(p)):
        sc, fl, rr = oracle.align(p.read(i), p.target(i), pen, limit=oracle.limit_for(pen, 3))
        assert (s[i], f[i], list(runs[i])) == (sc, fl, list(rr)), i


def test_results_independent_of_batch_composition(aligner, gen_lib):
    """Each pair's result is the same alone, in a shuffled batch and with a small workspace."""
    p = gen.generate(gen.WFA_UNEVEN, 600)
    me = gen.per_pair_max_edits(gen.WFA_UNEVEN, p)
    full = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, aligner=aligner)
    perm = np.random.default_rng(9).permutation(len(p))
    sub = gen.generate(gen.WFA_UNEVEN, index=perm)
    shuf = device_results(sub, "wfa", AFF, int(me.max()), per_pair=me[perm], max_length=1000, workspace=64 << 20)
    for j, i in enumerate(perm):
        assert shuf[0][j] == full[0][i] and shuf[1][j] == full[1][i]
        assert np.array_equal(shuf[2][j], full[2][i])


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32, 256])
def test_wfa_every_group_size_matches_oracle(aligner, oracle_lib, gen_lib, lanes):
    """Lanes per pair change only the schedule, never a result."""
    import paper_2208_01243_gb300 as aim
    w = gen.WFA_UNEVEN
    p = gen.concat([gen.generate(gen.WFA_150BP, 1_203), gen.generate(w, 301)])
    me = np.concatenate([np.full(1_203, 6, np.int32), gen.per_pair_max_edits(w, p)[1_203:]])
    lim = np.array([oracle.limit_for(AFF, int(k)) for k in me], np.int64)
    orc = oracle_results(p, AFF, lim)
    aim.aim_set_wfa_group(aligner.ctx, lanes)
    try:
        dev = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, aligner=aligner)
    finally:
        aim.aim_set_wfa_group(aligner.ctx, 0)
    assert_same(dev, orc, what=f"wfa lanes={lanes}")


LONG = gen.Workload("long_2000_4000bp_2_10pct", 6, 0, 2000, 4000, 0.02, 0.10, 0.0, "wfa", AFF, None,
                    max_edits_frac=0.10)


@pytest.mark.parametrize("lanes", [0, 32, 256])
def test_long_reads_match_oracle(aligner, oracle_lib, gen_lib, lanes):
    """Long, noisy pairs (2-4 kbp, up to 10 % edits): the default (block-wide groups) and warp groups agree with the oracle."""
    import paper_2208_01243_gb300 as aim
    p = gen.generate(LONG, 24)
    me = gen.per_pair_max_edits(LONG, p)
    orc = oracle_results(p, AFF, np.array([oracle.limit_for(AFF, int(k)) for k in me], np.int64))
    aim.aim_set_wfa_group(aligner.ctx, lanes)
    try:
        dev = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, aligner=aligner)
    finally:
        aim.aim_set_wfa_group(aligner.ctx, 0)
    assert_same(dev, orc, what=f"long reads lanes={lanes}")


def test_reads_beyond_10kbp_exact_score(aligner, oracle_lib, gen_lib):
    """20-31 kbp pairs at 1-2 % edits (past the serving workload's 10 kbp): score, flags and the canonical CIGAR
    equal the row-block oracle's (the full matrix would not fit), and the CIGAR re-costs to the score."""
    w = gen.Workload("wfa_20_31kbp_1_2pct", 91, 6, 20_000, 31_000, 0.01, 0.02, 0.0, "wfa", AFF, None,
                     max_edits_frac=0.02)
    p = gen.generate(w)
    me = gen.per_pair_max_edits(w, p)
    dev = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, aligner=aligner)
    lim = np.array([oracle.limit_for(AFF, int(k)) for k in me], np.int64)
    s, f, off, cig, lens = oracle.align_batch(p, AFF, lim, rows_per_block=0)
    assert_same(dev, (s, f, [cig[off[i]:off[i] + lens[i]].astype(np.uint32) for i in range(len(p))]),
                what="20-31 kbp")
    for i in range(len(p)):
        assert cost(decode(dev[2][i]), p.read(i), p.target(i), AFF) == dev[0][i]


@pytest.mark.parametrize("algo,pen,band", [("gotoh", (0, 3, 0, 4), -1),       # NW linear gap, x=3, e=4 (Section 2.4.1)
                                           ("gotoh", (0, 3, 4, 1), -1),       # SWG, x=3, o=4, e=1 (Section 2.4.2)
                                           ("wfa", (0, 3, 4, 1), -1)])        # WFA, x=3, o=4, e=1 (Section 2.4.4)
def test_paper_cost_schemes(aligner, oracle_lib, gen_lib, algo, pen, band):
    """The paper's own costs on 150 bp pairs at 4 % edits (max_edits 6)."""
    p = gen.generate(gen.WFA_150BP, 5_003)
    lim = np.full(len(p), oracle.limit_for(pen, 6), np.int64)
    orc = oracle_results(p, pen, lim, band=band)
    dev = device_results(p, algo, pen, 6, band=band, aligner=aligner)
    assert_same(dev, orc, what=f"{algo} {pen}")


def _adaptive_oracle(p, pen, lim, min_len, max_dist):
    s, f, off, cig, lens = oracle.wfa_adaptive_batch(p, pen, lim, min_len=min_len, max_dist=max_dist)
    return s, f, [cig[off[i]:off[i] + lens[i]].astype(np.uint32) for i in range(len(p))]


@pytest.mark.parametrize("params", [(10, 50), (4, 5), (2, 1)])
@pytest.mark.parametrize("lanes", [0, 4, 32, 256])
def test_wfa_adaptive_matches_its_oracle(aligner, oracle_lib, gen_lib, params, lanes):
    """WFA-adaptive (pruning + source-following traceback) equals the step-by-step CPU heuristic bit for bit."""
    import paper_2208_01243_gb300 as aim
    pu = gen.generate(gen.WFA_UNEVEN, 400)
    ps = gen.generate(gen.WFA_150BP, 1_001)
    p = gen.concat([pu, ps])
    me = np.concatenate([gen.per_pair_max_edits(gen.WFA_UNEVEN, pu), np.full(len(ps), 6, np.int32)])
    lim = np.array([oracle.limit_for(AFF, int(k)) for k in me], np.int64)
    orc = _adaptive_oracle(p, AFF, lim, *params)
    aim.aim_set_wfa_adaptive(aligner.ctx, *params)
    aim.aim_set_wfa_group(aligner.ctx, lanes)
    try:
        dev = device_results(p, "wfa_adaptive", AFF, int(me.max()), per_pair=me, aligner=aligner)
    finally:
        aim.aim_set_wfa_group(aligner.ctx, 0)
        aim.aim_set_wfa_adaptive(aligner.ctx, 10, 50)
    assert_same(dev, orc, what=f"wfa adaptive {params} lanes={lanes}")


def test_wfa_adaptive_paper_costs_150bp(aligner, oracle_lib, gen_lib):
    """The paper's Table 3 setting in shape: 150 bp, 2 % edits, costs x=3 o=4 e=1 (Section 2.4.4)."""
    w = gen.Workload("wfa_adaptive_150bp_2pct", 7, 0, 150, 150, 0.02, 0.02, 0.0, "wfa_adaptive", (0, 3, 4, 1), 3)
    p = gen.generate(w, 3_001)
    pen = (0, 3, 4, 1)
    lim = np.full(len(p), oracle.limit_for(pen, 3), np.int64)
    orc = _adaptive_oracle(p, pen, lim, 10, 50)
    dev = device_results(p, "wfa_adaptive", pen, 3, aligner=aligner)
    assert_same(dev, orc, what="wfa adaptive 150bp paper costs")
    exact = oracle_results(p, pen, lim)
    assert (dev[0] == exact[0]).mean() > 0.99


@pytest.mark.parametrize("lanes", [0, 1, 4, 32, 256])
def test_wfa_adaptive_hand_worked_pruning(aligner, oracle_lib, lanes):
    """The hand-worked pruning cases (tests/golden/adaptive_prune.txt) through the CUDA kernel: score, flags and ops."""
    import paper_2208_01243_gb300 as aim
    from test_oracle_adaptive import GOLDEN_ROWS
    aim.aim_set_wfa_group(aligner.ctx, lanes)
    try:
        for r, t, pen, lim, lmin, dmax, score, ops, kept in GOLDEN_ROWS:
            p = gen.from_strings([r.decode()], [t.decode()])
            aim.aim_set_wfa_adaptive(aligner.ctx, lmin, dmax)
            dev = device_results(p, "wfa_adaptive", pen, -1, max_score=lim, aligner=aligner)
            if score < 0:
                assert (dev[0][0], dev[1][0]) == (-1, oracle.F_REJECTED), (r, t)
            else:
                assert (dev[0][0], dev[1][0], decode(dev[2][0])) == (score, 0, ops), (r, t, lanes)
    finally:
        aim.aim_set_wfa_group(aligner.ctx, 0)
        aim.aim_set_wfa_adaptive(aligner.ctx, 10, 50)


@pytest.mark.parametrize("algo,band", [("edit", 6), ("edit", 10), ("gotoh", 7), ("gotoh", 12)])
def test_dp_several_pairs_per_warp(oracle_lib, gen_lib, algo, band):
    """Narrow bands run 4 (band <= 7) or 2 (band <= 15) pairs per warp, one per segment of 8 or 16 lanes, each
    with its own length, early exit and deferred traceback slot; with 40 MiB, 320 MiB and 4 GiB of workspace
    (one round of slots per flush up to 32 slots)."""
    w = gen.WFA_150BP
    p = gen.generate(w, 12_007)
    pen = AFF if algo == "gotoh" else oracle.UNIT
    max_edits = band if algo == "edit" else 3
    lim = np.array([oracle.limit_for(pen, max_edits, unit=algo == "edit")] * len(p), np.int64)
    orc = oracle_results(p, pen, lim, band=band)
    assert ((orc[1] & oracle.F_REJECTED) > 0).sum() > 100 and (orc[1] == 0).sum() > 100
    for ws in (40 << 20, 320 << 20, 4 << 30):
        dev = device_results(p, algo, pen, max_edits, band=band, workspace=ws)
        assert_same(dev, orc, what=f"{algo} band {band} workspace={ws >> 20} MiB")
