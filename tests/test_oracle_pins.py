"""Pins for the CPU oracle: brute force, closed forms, hand-worked examples.

None of these re-types the oracle's recurrences: brute force prices every op
string by the closed-form cost, the closed forms follow from the cost model,
and the hand-worked examples were derived by hand (tests/golden).
"""
import itertools
import os
import random

import pytest

import oracle
from oracle import brute
from oracle.cigar import cost, decode, encode

SCHEMES = [(0, 4, 6, 2), (0, 3, 4, 1), (0, 1, 0, 1), (0, 2, 1, 1), (0, 1, 2, 3), (0, 5, 1, 1)]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        r, t, u, a, ops = line.split()
        rows.append((r.encode(), t.encode(), int(u), int(a), ops))
    return rows


@pytest.mark.parametrize("scheme", SCHEMES)
def test_exhaustive_tiny_binary_alphabet(oracle_lib, scheme):
    """Every read/target over {A, C} with lengths 0..3, unbanded and banded."""
    n_checked = 0
    for L1 in range(4):
        for L2 in range(4):
            for r in itertools.product(b"AC", repeat=L1):
                for t in itertools.product(b"AC", repeat=L2):
                    r_, t_ = bytes(r), bytes(t)
                    for band in (-1, 0, 1):
                        bs, bops = brute.best(r_, t_, scheme, band)
                        s, fl, runs = oracle.align(r_, t_, scheme, band=band)
                        if bs is None:
                            assert fl & oracle.F_REJECTED and s == -1
                        else:
                            assert (s, decode(runs)) == (bs, bops), (r_, t_, scheme, band)
                        n_checked += 1
    assert n_checked == 3 * sum(2 ** a * 2 ** b for a in range(4) for b in range(4))


def test_random_tiny_dna(oracle_lib):
    rnd = random.Random(7)
    for _ in range(600):
        L1, L2 = rnd.randint(0, 5), rnd.randint(0, 5)
        if L1 + L2 > 9:
            continue
        r = bytes(rnd.choice(b"ACGT") for _ in range(L1))
        t = bytes(rnd.choice(b"ACGT") for _ in range(L2))
        sc = rnd.choice(SCHEMES)
        band = rnd.choice([-1, -1, 1, 2])
        bs, bops = brute.best(r, t, sc, band)
        s, fl, runs = oracle.align(r, t, sc, band=band)
        if bs is None:
            assert fl & oracle.F_REJECTED
        else:
            assert (s, decode(runs)) == (bs, bops), (r, t, sc, band)


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"{r[0].decode()}-{r[1].decode()}")
def test_hand_worked(oracle_lib, row):
    r, t, unit, affine, ops = row
    s, fl, runs = oracle.align(r, t, oracle.UNIT)
    assert s == unit and fl == 0
    assert cost(decode(runs), r, t, oracle.UNIT) == unit
    s, fl, runs = oracle.align(r, t, (0, 4, 6, 2))
    assert (s, decode(runs)) == (affine, ops)
    # the fixtures themselves must agree with brute force where it is affordable
    if len(r) + len(t) <= 12:
        assert brute.best(r, t, (0, 4, 6, 2))[0] == affine
        assert brute.best(r, t, oracle.UNIT)[0] == unit


@pytest.mark.parametrize("n", [1, 5, 31, 32, 33, 100])
def test_closed_forms(oracle_lib, n):
    rnd = random.Random(n)
    s = bytes(rnd.choice(b"ACGT") for _ in range(n))
    for sc in [(0, 4, 6, 2), oracle.UNIT, (0, 3, 4, 1)]:
        _, x, o, e = sc
        # identical pair: score 0, all matches
        assert oracle.align(s, s, sc)[0::2] == (0, encode("M" * n))
        # empty read: one n-base D; empty target: one n-base I
        assert oracle.align(b"", s, sc)[0::2] == (o + e * n, encode("D" * n))
        assert oracle.align(s, b"", sc)[0::2] == (o + e * n, encode("I" * n))
    assert oracle.align(b"", b"", (0, 4, 6, 2))[0::2] == (0, [])
    # all-mismatch pair of equal length: n*x when n*x <= 2*(o+e*n)
    a, c = b"A" * n, b"C" * n
    assert oracle.align(a, c, oracle.UNIT)[0::2] == (n, encode("X" * n))
    assert oracle.align(a, c, (0, 4, 6, 2))[0::2] == (4 * n, encode("X" * n))


def test_unit_cost_equals_textbook_levenshtein(oracle_lib):
    rnd = random.Random(3)
    for _ in range(300):
        r = bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 60)))
        t = bytes(rnd.choice(b"ACGT") for _ in range(rnd.randint(0, 60)))
        assert oracle.align(r, t, oracle.UNIT, cigar=False)[0] == oracle.levenshtein(r, t)


def test_levenshtein_known_values(oracle_lib):
    # textbook values
    assert oracle.levenshtein(b"", b"") == 0
    assert oracle.levenshtein(b"ACGT", b"") == 4
    assert oracle.levenshtein(b"GATTACA", b"GCATTAC") == 2
    assert oracle.levenshtein(b"AAAA", b"CCCC") == 4
    assert oracle.levenshtein(b"ACGT", b"TGCA") == 4


def test_threshold_reject(oracle_lib):
    r, t = b"GATTACA", b"GCATTAC"
    assert oracle.align(r, t, (0, 4, 6, 2), limit=16)[0] == 16
    s, fl, runs = oracle.align(r, t, (0, 4, 6, 2), limit=15)
    assert (s, fl, runs) == (-1, oracle.F_REJECTED, [])
    # band narrower than |n-m| rejects outright
    assert oracle.align(b"A", b"AAA", (0, 4, 6, 2), band=1)[1] == oracle.F_REJECTED


def test_limit_reading():
    assert oracle.limit_for((0, 4, 6, 2), 6) == 48
    assert oracle.limit_for(oracle.UNIT, 10, unit=True) == 10
    assert oracle.limit_for((0, 4, 6, 2), 6, max_score=30) == 30
    assert oracle.limit_for((0, 9, 1, 1), 3) == 27


def test_pack_layout_closed_forms():
    from oracle import pack
    assert pack.pack_one(b"A" * 32) == [0]
    assert pack.pack_one(b"T" * 32) == [0xFFFFFFFFFFFFFFFF]
    assert pack.pack_one(b"C") == [1 << 62]
    assert pack.pack_one(b"ACGT") == [0x1B << 56]
    assert pack.pack_one(b"A" * 32 + b"G") == [0, 2 << 62]
    assert pack.pack_one(b"") == []
    with pytest.raises(ValueError):
        pack.pack_one(b"ACGN")
