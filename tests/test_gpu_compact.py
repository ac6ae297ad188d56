"""Compact wavefront histories (exact WFA, 32-lane and whole-block groups, reads longer than 2,048 bp): the
forward pass keeps the last few wavefronts in a live ring and the history one 16-bit word (reads up to 16,382 bp)
or 32-bit word (longer) per entry, M~ plus two source bits from which the traceback rebuilds I~ and D~.  The
results must equal the oracle's bit for bit: canonical CIGARs included, on many short pairs run through the
compact forms (a max_length above the thresholds selects them), on 2-10 kbp pairs, and on pairs beyond the
32,000 bp that the 8-byte form's int16 offsets allowed."""
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
    a = aim.Aligner(0, 8 << 30)
    yield a
    a.close()


@pytest.mark.parametrize("max_length", [3000, 20000])         # 16-bit and 32-bit compact words
@pytest.mark.parametrize("lanes", [32, 256])
def test_compact_forms_on_many_pairs(aligner, oracle_lib, gen_lib, max_length, lanes):
    """4,003 pairs of 150-1000 bp (the uneven workload's shapes) and 150 bp pairs with 10 % unrelated targets,
    through the compact forms (max_length above 2,048 or 16,382 bp selects them)."""
    import paper_2208_01243_gb300 as aim
    pu = gen.generate(gen.WFA_UNEVEN, 2_001)
    ps = gen.generate(gen.WFA_150BP, 2_002)
    p = gen.concat([pu, ps])
    me = np.concatenate([gen.per_pair_max_edits(gen.WFA_UNEVEN, pu), np.full(len(ps), 6, np.int32)])
    lim = np.array([oracle.limit_for(AFF, int(k)) for k in me], np.int64)
    orc = oracle_results(p, AFF, lim)
    aim.aim_set_wfa_group(aligner.ctx, lanes)
    try:
        dev = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, max_length=max_length, aligner=aligner)
    finally:
        aim.aim_set_wfa_group(aligner.ctx, 0)
    assert_same(dev, orc, what=f"compact max_length={max_length} lanes={lanes}")


def test_compact_banded(aligner, oracle_lib, gen_lib):
    """Band 25 on the 250 bp workload's pairs through the 16-bit compact form."""
    import paper_2208_01243_gb300 as aim
    w = gen.GOTOH_WFA_250BP
    p = gen.generate(w, 2_001)
    orc = oracle_results(p, AFF, limits(w, p), band=25)
    aim.aim_set_wfa_group(aligner.ctx, 32)
    try:
        dev = device_results(p, "wfa", AFF, 25, band=25, max_length=4000, aligner=aligner)
    finally:
        aim.aim_set_wfa_group(aligner.ctx, 0)
    assert_same(dev, orc, what="compact banded")


LONG = gen.Workload("long_2000_10000bp_1_10pct", 61, 0, 2000, 10000, 0.01, 0.10, 0.0, "wfa", AFF, None,
                    max_edits_frac=0.10)


@pytest.mark.parametrize("lanes", [0, 32])
def test_long_pairs_canonical(aligner, oracle_lib, gen_lib, lanes):
    """40 pairs of 2-10 kbp at 1-10 % edits (the default picks whole-block groups for most), against the
    row-block oracle."""
    import paper_2208_01243_gb300 as aim
    p = gen.generate(LONG, 40)
    me = gen.per_pair_max_edits(LONG, p)
    orc = oracle_results_rows(p, AFF, np.array([oracle.limit_for(AFF, int(k)) for k in me], np.int64))
    aim.aim_set_wfa_group(aligner.ctx, lanes)
    try:
        dev = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, aligner=aligner)
    finally:
        aim.aim_set_wfa_group(aligner.ctx, 0)
    assert_same(dev, orc, what=f"2-10 kbp lanes={lanes}")
    assert (dev[1] == 0).sum() >= 30


def oracle_results_rows(p, penalties, lim, band=-1):
    s, f, off, cig, lens = oracle.align_batch(p, penalties, lim, band=band, rows_per_block=0)
    return s, f, [cig[off[i]:off[i] + lens[i]].astype(np.uint32) for i in range(len(p))]


def test_reads_beyond_32kbp(aligner, oracle_lib, gen_lib):
    """Two pairs of 32.5-34 kbp at 0.5-1 % edits (past the int16 offsets' 32,000 bp): the 32-bit compact form,
    canonical CIGARs against the row-block oracle (about 2 x 10^9 cell updates per pair on the host)."""
    w = gen.Workload("wfa_32_34kbp", 62, 0, 32_500, 34_000, 0.005, 0.01, 0.0, "wfa", AFF, None,
                     max_edits_frac=0.01)
    p = gen.generate(w, 2)
    me = gen.per_pair_max_edits(w, p)
    orc = oracle_results_rows(p, AFF, np.array([oracle.limit_for(AFF, int(k)) for k in me], np.int64))
    dev = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, aligner=aligner)
    assert_same(dev, orc, what="33-40 kbp")
    assert (dev[1] == 0).all()
    for i in range(len(p)):
        assert cost(decode(dev[2][i]), p.read(i), p.target(i), AFF) == dev[0][i]
