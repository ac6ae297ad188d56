"""Pins for the windowed GenASM oracle (Section 2.4.3, our reading).

Inside one window (both sequences no longer than W) the method is exact: the
score must be the edit distance (brute force and the separate Levenshtein
routine) and the CIGAR the first optimal op string in the traceback order,
found by enumerating every op string.  Across windows it is a heuristic: the
hand-worked examples in tests/golden/genasm_windows.txt fix the window rule,
closed forms fix the special cases, and at any size the CIGAR must be a valid
alignment whose edit count is the score, never below the edit distance.
"""
import itertools
import os
import random

import numpy as np
import pytest

import gen
import oracle
from oracle import brute
from oracle.cigar import cost, decode, reconstruct_target

UNIT = (0, 1, 0, 1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "genasm_windows.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        r, t, w, o, k, s, ops = line.split()
        rows.append((r.encode(), t.encode(), int(w), int(o), int(k), int(s), ops))
    return rows


def test_one_window_equals_brute_force_binary(oracle_lib):
    """Every read/target over {A, C} of lengths 0..4: score and CIGAR from enumeration."""
    for L1 in range(5):
        for L2 in range(5):
            if L1 + L2 > 8:
                continue
            for r in itertools.product(b"AC", repeat=L1):
                for t in itertools.product(b"AC", repeat=L2):
                    r_, t_ = bytes(r), bytes(t)
                    bs, bops = brute.genasm_first(r_, t_)
                    for W in sorted({max(L1, L2, 1), 64}):
                        s, f, runs = oracle.genasm(r_, t_, W=W, O=W - 1 if W > 1 else 0)
                        assert f == 0 and (s, decode(runs)) == (bs, bops), (r_, t_, W)


def test_one_window_equals_brute_force_dna(oracle_lib):
    rnd = random.Random(11)
    for _ in range(400):
        L1, L2 = rnd.randint(0, 5), rnd.randint(0, 5)
        if L1 + L2 > 9:
            continue
        r = bytes(rnd.choice(b"ACGT") for _ in range(L1))
        t = bytes(rnd.choice(b"ACGT") for _ in range(L2))
        bs, bops = brute.genasm_first(r, t)
        s, f, runs = oracle.genasm(r, t)
        assert (s, decode(runs)) == (bs, bops), (r, t)


def test_one_window_score_is_levenshtein(oracle_lib, gen_lib):
    """Generated pairs up to 64 bp (one window at W=64): the score is the textbook edit distance."""
    w = gen.Workload("genasm_pin_short", 71, 300, 20, 48, 0.0, 0.3, 0.1, "genasm", UNIT, None)
    p = gen.generate(w)
    for i in range(len(p)):
        r, t = p.read(i), p.target(i)
        assert max(len(r), len(t)) <= 64
        s, f, runs = oracle.genasm(r, t)
        assert s == oracle.levenshtein(r, t)
        assert cost(decode(runs), r, t, UNIT) == s


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"{r[0].decode()}-{r[1].decode()}-W{r[2]}-k{r[4]}")
def test_hand_worked_windows(oracle_lib, row):
    r, t, W, O, k, score, ops = row
    s, f, runs = oracle.genasm(r, t, k=k, W=W, O=O)
    if score < 0:
        assert (s, f, runs) == (-1, oracle.F_REJECTED, [])
    else:
        assert (s, f, decode(runs)) == (score, 0, ops)


@pytest.mark.parametrize("W,O", [(64, 24), (16, 4), (4, 1), (1, 0)])
def test_closed_forms(oracle_lib, W, O):
    rnd = random.Random(W)
    seq = bytes(rnd.choice(b"ACGT") for _ in range(300))
    assert oracle.genasm(seq, seq, W=W, O=O)[:2] == (0, 0)
    assert decode(oracle.genasm(seq, seq, W=W, O=O)[2]) == "M" * 300
    # nothing in common: every read base is a mismatch (X before I and D), in every window
    s, f, runs = oracle.genasm(b"A" * 200, b"C" * 200, W=W, O=O)
    assert (s, decode(runs)) == (200, "X" * 200)
    assert oracle.genasm(b"A" * 200, b"C" * 200, k=199, W=W, O=O)[:2] == (-1, oracle.F_REJECTED)
    # empty sides: one gap
    assert (oracle.genasm(b"", seq[:77], W=W, O=O)[0], decode(oracle.genasm(b"", seq[:77], W=W, O=O)[2])) == (77, "D" * 77)
    assert (oracle.genasm(seq[:5], b"", W=W, O=O)[0], decode(oracle.genasm(seq[:5], b"", W=W, O=O)[2])) == (5, "IIIII")
    assert oracle.genasm(b"", b"", W=W, O=O)[:3] == (0, 0, [])


def test_threshold_rule(oracle_lib):
    """One window: accepted iff the edit distance is at most k."""
    rnd = random.Random(3)
    for _ in range(200):
        r = bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 40)))
        t = bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 40)))
        ed = oracle.levenshtein(r, t)
        assert oracle.genasm(r, t, k=ed)[0] == ed
        if ed:
            assert oracle.genasm(r, t, k=ed - 1)[:3] == (-1, oracle.F_REJECTED, [])


@pytest.mark.parametrize("length,rate", [(150, 0.05), (1000, 0.05), (1000, 0.15)])
def test_windowed_alignments_are_valid(oracle_lib, gen_lib, length, rate):
    """Any size: a valid alignment of the reported edit count, never below the edit distance."""
    w = gen.Workload("genasm_pin_long", 72, 60, length, length, rate, rate, 0.1, "genasm", UNIT, None)
    p = gen.generate(w)
    worse = 0
    for i in range(len(p)):
        r, t = p.read(i), p.target(i)
        s, f, runs = oracle.genasm(r, t)
        ops = decode(runs)
        assert f == 0
        assert cost(ops, r, t, UNIT) == s
        rec = reconstruct_target(ops, r)
        assert rec is not None and len(rec) == len(t)
        assert all(a == ord("?") or a == b for a, b in zip(rec, t))
        ed = oracle.levenshtein(r, t)
        assert s >= ed
        worse += s > ed
    assert worse < len(p)   # windows lose little on similar pairs


def test_threshold_is_the_windowed_edit_count(oracle_lib, gen_lib):
    """Rejected iff the windowed alignment has more than k edits: the early exit on a window whose distance
    exceeds the edits left changes no outcome, and k never changes an accepted result."""
    w = gen.Workload("genasm_pin_budget", 73, 80, 150, 400, 0.02, 0.1, 0.1, "genasm", UNIT, None)
    p = gen.generate(w)
    for i in range(len(p)):
        r, t = p.read(i), p.target(i)
        free = oracle.genasm(r, t)
        for k in range(max(free[0] - 3, 0), free[0] + 3):
            s, f, runs = oracle.genasm(r, t, k=k)
            if k < free[0]:
                assert (s, f, runs) == (-1, oracle.F_REJECTED, [])
            else:
                assert (s, f, runs) == free


def test_batch_matches_single(oracle_lib, gen_lib):
    w = gen.Workload("genasm_pin_batch", 74, 50, 50, 300, 0.0, 0.1, 0.2, "genasm", UNIT, None)
    p = gen.generate(w)
    lim = np.full(len(p), 12, np.int64)
    sc, fl, off, cig, lens = oracle.genasm_batch(p, lim, threads=3)
    for i in range(len(p)):
        s, f, runs = oracle.genasm(p.read(i), p.target(i), k=12)
        assert (sc[i], fl[i]) == (s, f)
        assert [int(v) for v in cig[off[i]:off[i] + lens[i]]] == runs
