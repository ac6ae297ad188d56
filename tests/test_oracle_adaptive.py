"""Pins for the step-by-step WFA-adaptive oracle.

With pruning off it is the exact WFA: its score must equal the brute-force
optimum and the full-matrix DP optimum, and its CIGAR must be a valid alignment
that re-costs to that score.  With pruning on it is a heuristic: its CIGAR must
still be a valid alignment re-costing to its score, the score can only be at
least the optimum, and similar pairs lose nothing.
"""
import itertools
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
