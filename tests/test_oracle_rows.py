"""Pins for the row-block form of the oracle (long pairs, memory linear in the target length per block).

It runs the same DP and the same canonical backward greedy as the full-matrix oracle, which brute force, closed
forms and hand-worked examples pin; here it must give the full-matrix oracle's score, flags and CIGAR on every
pair, for block sizes from one row to more than the read, with and without a band and a threshold.
"""
import itertools
import random

import numpy as np
import pytest

import gen
import oracle
from oracle.cigar import cost, decode

SCHEMES = [(0, 4, 6, 2), (0, 1, 0, 1), (0, 3, 4, 1), (0, 3, 0, 4)]


def test_tiny_pairs_every_block_size(oracle_lib):
    for L1 in range(4):
        for L2 in range(4):
            for r in itertools.product(b"AC", repeat=L1):
                for t in itertools.product(b"AC", repeat=L2):
                    r_, t_ = bytes(r), bytes(t)
                    for pen in SCHEMES:
                        for band in (-1, 1):
                            want = oracle.align(r_, t_, pen, band=band)
                            for K in (1, 2, 3, 5, 0):
                                assert oracle.align_rows(r_, t_, pen, band=band, rows_per_block=K) == want, \
                                    (r_, t_, pen, band, K)


@pytest.mark.parametrize("pen", SCHEMES)
def test_random_pairs_up_to_1kbp(oracle_lib, pen):
    rnd = random.Random(sum(pen))
    for it in range(60):
        n = rnd.choice([0, 1, 7, 31, 32, 33, 150, 400, 1000])
        r = bytes(rnd.choice(b"ACGT") for _ in range(n))
        t = bytearray(r)
        for _ in range(rnd.randint(0, max(1, n // 8))):
            op, pos = rnd.randint(0, 2), rnd.randint(0, len(t))
            if op == 0 and pos < len(t):
                t[pos] = rnd.choice(b"ACGT")
            elif op == 1:
                t.insert(pos, rnd.choice(b"ACGT"))
            elif pos < len(t):
                del t[pos]
        t = bytes(t)
        band = rnd.choice([-1, -1, 5, 40])
        limit = rnd.choice([1 << 62, 1 << 62, 30, 200])
        want = oracle.align(r, t, pen, band=band, limit=limit)
        for K in (1, 7, 0, 2000):
            got = oracle.align_rows(r, t, pen, band=band, limit=limit, rows_per_block=K)
            assert got == want, (n, len(t), pen, band, limit, K)


def test_batch_on_generated_long_pairs(oracle_lib, gen_lib):
    """Serving-shaped pairs up to 1 kbp (log-uniform lengths, 1-10 % edits, thresholds at 10 % of the length):
    the batch driver's row-block mode equals the full-matrix batch, element by element."""
    w = gen.Workload("rows_pin_100_1000bp", 81, 0, 100, 1000, 0.01, 0.10, 0.05, "wfa", (0, 4, 6, 2), None,
                     max_edits_frac=0.10)
    p = gen.generate(w, 120)
    me = gen.per_pair_max_edits(w, p)
    lim = np.array([oracle.limit_for((0, 4, 6, 2), int(k)) for k in me], np.int64)
    a = oracle.align_batch(p, (0, 4, 6, 2), lim, threads=4)
    b = oracle.align_batch(p, (0, 4, 6, 2), lim, threads=4, rows_per_block=0)
    c = oracle.align_batch(p, (0, 4, 6, 2), lim, threads=4, rows_per_block=13)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    assert (a[1] & oracle.F_REJECTED).sum() > 0 and (a[1] == 0).sum() > 0


def test_long_pair_is_valid_and_within_the_script_cost(oracle_lib, gen_lib):
    """One 5 kbp pair (the full matrix would take 300 MB): a valid alignment, re-costing to the score, no worse
    than the generator's own edit script."""
    w = gen.Workload("rows_pin_5kbp", 82, 0, 5000, 5000, 0.03, 0.03, 0.0, "wfa", (0, 4, 6, 2), None,
                     max_edits_frac=0.10)
    p = gen.generate(w, 1)
    s, f, runs = oracle.align_rows(p.read(0), p.target(0), (0, 4, 6, 2))
    assert f == 0 and cost(decode(runs), p.read(0), p.target(0), (0, 4, 6, 2)) == s
    assert s <= gen.script_cost_bound(p, 4, 6, 2)[0]
