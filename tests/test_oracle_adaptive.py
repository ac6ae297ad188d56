"""Pins for the step-by-step WFA-adaptive oracle.

With pruning off it is the exact WFA: its score must equal the brute-force
optimum and the full-matrix DP optimum, and its CIGAR must be a valid alignment
that re-costs to that score.  With pruning on it is a heuristic: its CIGAR must
still be a valid alignment re-costing to its score, the score can only be at
least the optimum, and similar pairs lose nothing.
"""
import itertools
import os
import random

import numpy as np
import pytest

import gen
import oracle
from oracle import brute
from oracle.cigar import cost, decode

SCHEMES = [(0, 4, 6, 2), (0, 3, 4, 1), (0, 1, 0, 1), (0, 2, 1, 1), (0, 1, 2, 3)]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_unpruned_equals_brute_force_optimum(oracle_lib, scheme):
    for L1 in range(4):
        for L2 in range(4):
            for r in itertools.product(b"AC", repeat=L1):
                for t in itertools.product(b"AC", repeat=L2):
                    r_, t_ = bytes(r), bytes(t)
                    for band in (-1, 1):
                        bs, _ = brute.best(r_, t_, scheme, band)
                        s, f, runs = oracle.wfa_adaptive(r_, t_, scheme, band=band, min_len=-1)
                        if bs is None:
                            assert f & oracle.F_REJECTED
                            continue
                        assert s == bs, (r_, t_, scheme, band)
                        assert cost(decode(runs), r_, t_, scheme) == s


def test_unpruned_equals_dp_on_generated_pairs(oracle_lib, gen_lib):
    p = gen.generate(gen.WFA_UNEVEN, 120)
    me = gen.per_pair_max_edits(gen.WFA_UNEVEN, p)
    lim = np.array([oracle.limit_for((0, 4, 6, 2), int(k)) for k in me], np.int64)
    a = oracle.wfa_adaptive_batch(p, (0, 4, 6, 2), lim, min_len=-1)
    d = oracle.align_batch(p, (0, 4, 6, 2), lim)
    assert np.array_equal(a[0], d[0]) and np.array_equal(a[1], d[1])
    for i in range(len(p)):
        if a[1][i] == 0:
            assert cost(decode(a[3][a[2][i]:a[2][i] + a[4][i]]), p.read(i), p.target(i), (0, 4, 6, 2)) == a[0][i]


def test_pruned_is_valid_and_never_better_than_optimal(oracle_lib, gen_lib):
    rnd = random.Random(5)
    p = gen.concat([gen.generate(gen.WFA_UNEVEN, 150), gen.generate(gen.WFA_150BP, 150)])
    me = np.concatenate([gen.per_pair_max_edits(gen.WFA_UNEVEN, p)[:150], np.full(150, 6, np.int32)])
    lim = np.array([oracle.limit_for((0, 4, 6, 2), int(k)) for k in me], np.int64)
    for min_len, max_dist in [(10, 50), (4, 5), (2, 1)]:
        a = oracle.wfa_adaptive_batch(p, (0, 4, 6, 2), lim, min_len=min_len, max_dist=max_dist)
        d = oracle.align_batch(p, (0, 4, 6, 2), lim, cigar=False)
        for i in range(len(p)):
            if a[1][i] == 0:
                ops = decode(a[3][a[2][i]:a[2][i] + a[4][i]])
                assert cost(ops, p.read(i), p.target(i), (0, 4, 6, 2)) == a[0][i]
                assert d[1][i] == 0 and a[0][i] >= d[0][i]
            else:
                assert a[1][i] == oracle.F_REJECTED
    # the published-style setting loses nothing on similar pairs
    a = oracle.wfa_adaptive_batch(p, (0, 4, 6, 2), lim)
    related = ~p.unrelated.astype(bool)
    same = (a[0] == d[0])[related]
    assert same.mean() > 0.98


def test_huge_distance_threshold_is_exact(oracle_lib, gen_lib):
    p = gen.generate(gen.WFA_150BP, 200)
    lim = np.full(len(p), 48, np.int64)
    a = oracle.wfa_adaptive_batch(p, (0, 4, 6, 2), lim, min_len=10, max_dist=1 << 20)
    b = oracle.wfa_adaptive_batch(p, (0, 4, 6, 2), lim, min_len=-1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ---------------- the pruning step, pinned by hand-worked cases ----------------

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adaptive_prune.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        r, t, x, o, e, lim, lmin, dmax, score, ops, kept = line.split()
        kd = {}
        for item in kept.split(";"):
            s, rng = item.split(":")
            lo, hi = rng.split(",")
            kd[int(s)] = (int(lo), int(hi))
        rows.append((r.encode(), t.encode(), (0, int(x), int(o), int(e)), int(lim), int(lmin), int(dmax),
                     int(score), ops, kd))
    return rows


GOLDEN_ROWS = _golden()


def _limit(lim):
    return (1 << 40) if lim < 0 else lim


@pytest.mark.parametrize("row", GOLDEN_ROWS, ids=lambda r: f"{r[0].decode()}-{r[1].decode()}")
def test_hand_worked_pruning(oracle_lib, row):
    """Score, ops and the diagonal range kept at every score, as derived by hand (Section 2.4.4, our rule)."""
    r, t, pen, lim, lmin, dmax, score, ops, kept = row
    s, f, runs = oracle.wfa_adaptive(r, t, pen, limit=_limit(lim), min_len=lmin, max_dist=dmax)
    if score < 0:
        assert (s, f, runs) == (-1, oracle.F_REJECTED, [])
    else:
        assert (s, f, decode(runs)) == (score, 0, ops)
        assert cost(ops, r, t, pen) == score
    s2, f2, got = oracle.wfa_adaptive_kept(r, t, pen, limit=_limit(lim), min_len=lmin, max_dist=dmax)
    assert (s2, f2) == (s, f)
    assert got == kept


def test_hand_worked_cases_cover_the_heuristic(oracle_lib):
    """The cases include one pruned above its optimum and one rejected only because of pruning."""
    worse = rejected = 0
    for r, t, pen, lim, lmin, dmax, score, ops, kept in GOLDEN_ROWS:
        exact = oracle.wfa_adaptive(r, t, pen, limit=_limit(lim), min_len=-1)
        assert exact[1] == 0
        worse += score > exact[0]
        rejected += score < 0
    assert worse >= 1 and rejected >= 1


# Planted mistakes: each is a plausible slip in the pruning step, made in a copy of the oracle's source on the CPU;
# every one must change at least one hand-worked result.  (Pruning the wavefront that reaches the end is not among
# them: the end diagonal is at distance 0, the smallest, so it is always kept, and the traceback never reads the
# other diagonals of that wavefront; the rule skips it all the same.)
def _mutants(src):
    out = {}

    def sub(name, old, new, count=None):
        assert old in src and (count is None or src.count(old) == count), name
        out[name] = src.replace(old, new)

    sub("drop a diagonal exactly max_distance behind", "d - dmin <= dmax", "d - dmin < dmax", 2)
    sub("prune only wider than min_length", "vhi - vlo + 1 >= lmin", "vhi - vlo + 1 > lmin", 1)
    sub("distance as the smaller of the two remainders", "dv > dh ? dv : dh", "dv < dh ? dv : dh", 3)
    sub("trim the left end only", "while (b >= a) {", "while (0) {", 1)
    sub("read position taken as h", "(int64_t)n - (h - k)", "(int64_t)n - h", 1)
    sub("smallest distance from the first valid diagonal", "if (d < dmin) dmin = d;",
        "if (dmin == INT64_MAX) dmin = d;", 1)
    # distances at f0 instead of the extended offset
    old = "Mv[k - lo] = f0 >= 0 ? wfa_extend_plain(P, n, T, m, k, f0) : WNEG;"
    assert old in src
    s = src.replace(old, old + " F0v[k - lo] = f0;")
    s = s.replace("static int32_t gcd32", "static __thread int32_t F0v[1 << 16];\nstatic int32_t gcd32", 1)
    b0, b1 = s.index("if (found < 0 && lmin >= 0"), s.index("/* keep [vlo, vhi] */")
    blk = s[b0:b1]
    for v in ("k", "a", "b"):
        blk = blk.replace(f"Mv[{v} - lo]", f"F0v[{v} - lo]")
    out["distance at f0 instead of the extended offset"] = s[:b0] + blk + s[b1:]
    # every far diagonal dropped, not only the outer ones
    old = "            vlo = a; vhi = b;\n"
    assert old in src
    out["far interior diagonals dropped too"] = src.replace(old, old + (
        "            for (int32_t q = vlo + 1; q < vhi; ++q) { const int32_t hq = Mv[q - lo]; if (hq < 0) continue;"
        " const int64_t dv = (int64_t)n - (hq - q), dh = (int64_t)m - hq, d = dv > dh ? dv : dh;"
        " if (d - dmin > dmax) { Mv[q - lo] = WNEG; Iv[q - lo] = WNEG; Dv[q - lo] = WNEG; } }\n"))
    return out


def test_planted_pruning_mistakes_fail_a_pin(oracle_lib, tmp_path):
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(oracle.__file__), "aim_oracle.c")).read()
    i32, u32, i64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64
    for j, (name, text) in enumerate(_mutants(src).items()):
        c = tmp_path / f"mutant{j}.c"
        so = tmp_path / f"mutant{j}.so"
        c.write_text(text)
        subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", str(c), "-o", str(so), "-lpthread"])
        lib = ctypes.CDLL(str(so))
        lib.oracle_wfa_adaptive.argtypes = [ctypes.c_char_p, u32, ctypes.c_char_p, u32, i32, i32, i32, i32, i64,
                                            i32, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_uint8),
                                            ctypes.c_void_p, u32, ctypes.POINTER(u32)]
        caught = False
        for r, t, pen, lim, lmin, dmax, score, ops, kept in GOLDEN_ROWS:
            sc, fl, nc = ctypes.c_int32(), ctypes.c_uint8(), ctypes.c_uint32()
            cap = len(r) + len(t) + 1
            buf = np.zeros(cap, np.uint32)
            rc = lib.oracle_wfa_adaptive(r, len(r), t, len(t), pen[1], pen[2], pen[3], -1, _limit(lim), lmin, dmax,
                                         ctypes.byref(sc), ctypes.byref(fl), ctypes.c_void_p(buf.ctypes.data), cap,
                                         ctypes.byref(nc))
            got = (rc, sc.value, decode(buf[:nc.value]) if sc.value >= 0 else "-")
            caught |= got != (0, score, ops)
        assert caught, f"planted mistake not caught: {name}"
