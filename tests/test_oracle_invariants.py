"""Invariants of exact alignment checked on the oracle over generated pairs."""
import random

import numpy as np
import pytest

import gen
import oracle
from oracle.cigar import cost, decode, max_deviation, reconstruct_target

AFF = (0, 4, 6, 2)


def _rand(rnd, n):
    return bytes(rnd.choice(b"ACGT") for _ in range(n))


def test_edit_distance_metric_axioms(oracle_lib):
    rnd = random.Random(11)
    for _ in range(150):
        a, b, c = (_rand(rnd, rnd.randint(0, 40)) for _ in range(3))
        ab = oracle.align(a, b, oracle.UNIT)[0]
        ba = oracle.align(b, a, oracle.UNIT)[0]
        bc = oracle.align(b, c, oracle.UNIT)[0]
        ac = oracle.align(a, c, oracle.UNIT)[0]
        assert ab == ba
        assert ac <= ab + bc
        assert ab >= abs(len(a) - len(b))
        assert (ab == 0) == (a == b)


def test_affine_symmetry_and_gap_lower_bound(oracle_lib):
    rnd = random.Random(12)
    for _ in range(150):
        a, b = _rand(rnd, rnd.randint(0, 50)), _rand(rnd, rnd.randint(0, 50))
        s_ab, _, runs_ab = oracle.align(a, b, AFF)
        s_ba, _, runs_ba = oracle.align(b, a, AFF)
        assert s_ab == s_ba
        if len(a) != len(b):
            assert s_ab >= 6 + 2 * abs(len(a) - len(b))
        # swapping roles swaps I and D in SOME optimal alignment: the mirrored ops re-cost to the same score
        mirrored = decode(runs_ab).translate(str.maketrans("ID", "DI"))
        assert cost(mirrored, b, a, AFF) == s_ba


@pytest.mark.parametrize("w", [gen.EDIT_NW_100BP, gen.WFA_150BP, gen.GOTOH_WFA_250BP, gen.WFA_UNEVEN],
                         ids=lambda w: w.name)
def test_generated_pairs_invariants(oracle_lib, gen_lib, w):
    p = gen.generate(w, 120 if w.len_max <= 250 else 24)
    pen = w.penalties
    unit = w.algo == "edit"
    me = gen.per_pair_max_edits(w, p)
    lim = np.array([oracle.limit_for(pen, int(k), unit=unit) for k in me], np.int64)
    # unbanded, unlimited: the true optimum of each pair
    s_full, f_full, off, cig, lens = oracle.align_batch(p, pen, np.full(len(p), 1 << 62, np.int64))
    bound = gen.script_cost_bound(p, pen[1], pen[2], pen[3])
    for i in range(len(p)):
        r, t = p.read(i), p.target(i)
        ops = decode(cig[off[i]:off[i] + lens[i]])
        assert cost(ops, r, t, pen) == s_full[i]          # re-costs to the reported score
        rec = reconstruct_target(ops, r)
        assert rec is not None and len(rec) == len(t)
        assert all(x == y or x == ord("?") for x, y in zip(rec, t))   # rebuilds the target
        if bound[i] >= 0:
            assert s_full[i] <= bound[i]                  # never worse than the generator's script
    # thresholded (and banded where the workload bands): rejects exactly when the optimum exceeds the limit
    s_thr, f_thr, off2, cig2, lens2 = oracle.align_batch(p, pen, lim, band=w.band)
    for i in range(len(p)):
        if w.band < 0:
            assert bool(f_thr[i] & oracle.F_REJECTED) == (s_full[i] > lim[i])
            if not f_thr[i]:
                assert s_thr[i] == s_full[i]
                assert list(cig2[off2[i]:off2[i] + lens2[i]]) == list(cig[off[i]:off[i] + lens[i]])
        else:
            ops_full = decode(cig[off[i]:off[i] + lens[i]])
            if max_deviation(ops_full) <= w.band and s_full[i] <= lim[i]:
                # the unbanded canonical path fits the band: banded result is the same
                assert s_thr[i] == s_full[i]
                assert list(cig2[off2[i]:off2[i] + lens2[i]]) == list(cig[off[i]:off[i] + lens[i]])
            if not f_thr[i]:
                assert s_thr[i] >= s_full[i]
    if w.unrelated_frac == 0 and w.band < 0:
        # related pairs with at most max_edits edits are never rejected
        assert not (f_thr & oracle.F_REJECTED).any()


def test_unit_band_equal_to_threshold_is_exact(oracle_lib, gen_lib):
    """A path of cost <= k never leaves |h - v| <= k, so banding unit cost at the threshold changes nothing."""
    p = gen.generate(gen.EDIT_NW_100BP, 200)
    lim = np.full(len(p), 10, np.int64)
    a = oracle.align_batch(p, oracle.UNIT, lim)
    b = oracle.align_batch(p, oracle.UNIT, lim, band=10)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_generator_reproducible_by_index(gen_lib):
    w = gen.WFA_150BP
    whole = gen.generate(w, 50)
    some = gen.generate(w, index=np.array([3, 17, 42]))
    for j, i in enumerate([3, 17, 42]):
        assert some.read(j) == whole.read(i) and some.target(j) == whole.target(i)
    assert 0.05 < whole.unrelated.mean() < 0.2 or len(whole) < 100
