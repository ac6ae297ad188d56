"""Batched form (bucketed queues, autotuned lanes per pair, CUDA-graph replay) against the plain form and the oracle."""
import numpy as np
import pytest

import gen
import oracle
from devutil import assert_same, device_results, oracle_results

pytestmark = pytest.mark.gpu

AFF = (0, 4, 6, 2)


def _mixed(n_uneven=2_500, n_short=2_003):
    pu = gen.generate(gen.WFA_UNEVEN, n_uneven)
    ps = gen.generate(gen.WFA_150BP, n_short)
    p = gen.concat([pu, ps])
    me = np.concatenate([gen.per_pair_max_edits(gen.WFA_UNEVEN, pu), np.full(n_short, 6, np.int32)])
    return p, me


def _batched(p, me, autotune, runs=2, scratch=0, compact=0, passes=None, bound=0, bounds=None, band=-1):
    import torch
    import paper_2208_01243_gb300 as aim
    n = len(p)
    cap = p.read_len.astype(np.int64) + p.target_len.astype(np.int64) + 1
    coff = np.zeros(n + 1, np.int64); coff[1:] = np.cumsum(cap)
    reads, targets, ro, to, rl, tl, cd, pp = aim.upload(p.reads, p.targets, p.read_off, p.target_off, p.read_len,
                                                        p.target_len, coff, me.astype(np.int32))
    al = aim.Aligner(0, 1 << 30)
    aim.aim_set_batch_compact(al.ctx, compact)
    aim.aim_set_batch_bound(al.ctx, bound)
    dev = rl.device
    scores = torch.full((n,), -7, dtype=torch.int32, device=dev)
    flags = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    lens = torch.zeros(n, dtype=torch.int32, device=dev)
    cig = torch.zeros(int(coff[-1]), dtype=torch.int32, device=dev)
    ml = int(max(p.read_len.max(), p.target_len.max()))
    plan = aim.aim_batch_plan(al.ctx, reads, targets, ro, to, rl, tl, ml, aim.penalties(4, 6, 2, band=band),
                              int(me.max()), pp, scores, cig, cd, lens, flags, scratch_bytes=scratch,
                              autotune=autotune)
    groups, counts = aim.aim_batch_info(plan)
    if passes is not None:
        passes.append(aim.aim_batch_passes(plan))
    if bounds is not None:
        bounds.append(aim.aim_batch_bound_passes(plan))
    outs = []
    for _ in range(runs):
        scores.fill_(-7); flags.fill_(255)
        aim.aim_batch_run(plan)
        torch.cuda.synchronize()
        s = scores.cpu().numpy(); f = flags.cpu().numpy(); ln = lens.cpu().numpy().view(np.uint32)
        cg = cig.cpu().numpy().view(np.uint32)
        outs.append((s, f, [cg[coff[i]:coff[i] + ln[i]] for i in range(n)], ln))
    aim.aim_batch_destroy(plan)
    al.close()
    return outs, groups, counts


@pytest.mark.parametrize("autotune", [False, True])
def test_batched_equals_plain_and_oracle(oracle_lib, gen_lib, autotune):
    import __graft_entry__
    __graft_entry__.build()
    p, me = _mixed()
    outs, groups, counts = _batched(p, me, autotune)
    assert sum(counts) == len(p)
    assert all(g in (1, 2, 4, 8, 16, 32, 256) for g in groups)
    plain = device_results(p, "wfa", AFF, int(me.max()), per_pair=me)
    for o in outs:                       # every replay gives the plain form's results, bit for bit
        assert np.array_equal(o[0], plain[0]) and np.array_equal(o[1], plain[1])
        assert all(np.array_equal(x, y) for x, y in zip(o[2], plain[2]))
    idx = np.random.default_rng(4).choice(len(p), 400, replace=False)
    sub = gen.concat([gen.from_strings([p.read(i)], [p.target(i)]) for i in idx])
    lim = np.array([oracle.limit_for(AFF, int(me[i])) for i in idx], np.int64)
    assert_same(outs[-1], oracle_results(sub, AFF, lim), idx=idx, what="batched vs oracle")


@pytest.mark.parametrize("autotune", [False, True])
def test_compact_first_pass_gives_the_plain_results(oracle_lib, gen_lib, autotune):
    """Compact first passes forced on every bucket that allows one, with the fewest lanes that fit (so many pairs
    outgrow them): the second pass re-aligns exactly those, and every replay equals the plain form bit for bit."""
    import __graft_entry__
    __graft_entry__.build()
    p, me = _mixed(6_000, 2_003)
    passes = []
    outs, groups, counts = _batched(p, me, autotune, compact=1, passes=passes, scratch=4 << 30)
    first, full, n_compact = passes[0]
    assert n_compact > 0 and any(f and f < g for f, g in zip(first, full))
    plain = device_results(p, "wfa", AFF, int(me.max()), per_pair=me)
    for o in outs:
        assert (o[1] & 8).sum() == 0                 # no pair left flagged after the full pass
        assert np.array_equal(o[0], plain[0]) and np.array_equal(o[1], plain[1])
        assert all(np.array_equal(x, y) for x, y in zip(o[2], plain[2]))
    # never: one pass, the same results
    passes = []
    outs2, _, _ = _batched(p, me, autotune, runs=1, compact=2, passes=passes, scratch=4 << 30)
    assert passes[0][2] == 0
    assert np.array_equal(outs2[0][0], plain[0]) and np.array_equal(outs2[0][1], plain[1])


@pytest.mark.parametrize("autotune", [False, True])
@pytest.mark.parametrize("band", [-1, 25])
def test_bound_pass_gives_the_plain_results(oracle_lib, gen_lib, autotune, band):
    """Bound passes forced on every bucket: each exact pass runs with min(limit, bound) as its pairs' limit, and
    every replay equals the plain form (no bound pass) bit for bit, rejected pairs included (a tenth of the
    150 bp pairs are unrelated and exceed their limit); a sample also equals the oracle."""
    import __graft_entry__
    __graft_entry__.build()
    p, me = _mixed(3_000, 2_003)
    if band >= 0:
        keep = np.flatnonzero(np.abs(p.target_len.astype(np.int64) - p.read_len.astype(np.int64)) <= band)
        p = gen.concat([gen.from_strings([p.read(i)], [p.target(i)]) for i in keep])
        me = me[keep]
    bounds = []
    outs, groups, counts = _batched(p, me, autotune, bound=1, bounds=bounds, scratch=4 << 30, band=band)
    lanes, n_bound = bounds[0]
    assert n_bound >= 1 and all(g in (0, 4) for g in lanes)
    assert all(lanes[k] == 4 for k in range(32) if counts[k])
    plain = device_results(p, "wfa", AFF, int(me.max()), per_pair=me, band=band)
    assert (plain[1] & 1).sum() > 0                  # some pairs are rejected at their limit
    for o in outs:
        assert np.array_equal(o[0], plain[0]) and np.array_equal(o[1], plain[1])
        assert np.array_equal(o[3], plain[3])
        assert all(np.array_equal(x, y) for x, y in zip(o[2], plain[2]))
    idx = np.random.default_rng(9).choice(len(p), 300, replace=False)
    sub = gen.concat([gen.from_strings([p.read(i)], [p.target(i)]) for i in idx])
    lim = np.array([oracle.limit_for(AFF, int(me[i])) for i in idx], np.int64)
    assert_same(outs[-1], oracle_results(sub, AFF, lim, band=band), idx=idx, what="bound pass vs oracle")
    # never: no bound pass, the same results
    bounds = []
    outs2, _, _ = _batched(p, me, autotune, runs=1, bound=2, bounds=bounds, scratch=4 << 30, band=band)
    assert bounds[0][1] == 0
    assert np.array_equal(outs2[0][0], plain[0]) and np.array_equal(outs2[0][1], plain[1])


def test_tune_choices_export_and_import(gen_lib):
    """A plan made with autotune off in a context that imported another context's exported choices uses the same
    lanes, compact and bound passes per bucket, and gives the same results; a malformed text imports nothing."""
    import torch
    import paper_2208_01243_gb300 as aim
    p, me = _mixed(4_000, 1_003)
    n = len(p)
    cap = p.read_len.astype(np.int64) + p.target_len.astype(np.int64) + 1
    coff = np.zeros(n + 1, np.int64); coff[1:] = np.cumsum(cap)
    reads, targets, ro, to, rl, tl, cd, pp = aim.upload(p.reads, p.targets, p.read_off, p.target_off, p.read_len,
                                                        p.target_len, coff, me.astype(np.int32))
    ml = int(max(p.read_len.max(), p.target_len.max()))
    runs = []
    text = None
    for autotune in (True, False):
        al = aim.Aligner(0, 1 << 30)
        if text is not None:
            with pytest.raises(aim.AimError):
                aim.aim_tune_import(al.ctx, "4 6 2 -1 3 200 32 0\n")        # a field short
            assert aim.aim_tune_export(al.ctx) == ""
            aim.aim_tune_import(al.ctx, text)
            assert aim.aim_tune_export(al.ctx) == text
        out = al.outputs(n, cigar_capacity=torch.from_numpy(cap))
        out["cigars"].zero_()   # entries past a pair's runs are not written: compare whole buffers from zero
        plan = aim.aim_batch_plan(al.ctx, reads, targets, ro, to, rl, tl, ml, aim.penalties(4, 6, 2), int(me.max()),
                                  pp, out["scores"], out["cigars"], out["cigar_offsets"], out["cigar_lens"],
                                  out["flags"], autotune=autotune)
        aim.aim_batch_run(plan); torch.cuda.synchronize()
        runs.append((aim.aim_batch_info(plan)[0], aim.aim_batch_passes(plan)[:2], aim.aim_batch_bound_passes(plan)[0],
                     out["scores"].cpu().numpy().copy(), out["flags"].cpu().numpy().copy(),
                     out["cigars"].cpu().numpy().copy()))
        if autotune:
            text = aim.aim_tune_export(al.ctx)
            assert len(text.splitlines()) >= sum(1 for c in aim.aim_batch_info(plan)[1] if c)
        aim.aim_batch_destroy(plan)
        al.close()
    a, b = runs
    assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2]
    assert all(np.array_equal(x, y) for x, y in zip(a[3:], b[3:]))


def test_batched_replay_sees_new_contents(gen_lib):
    """The plan binds buffers, not data: a replay after the inputs change aligns the new pairs."""
    import torch
    import paper_2208_01243_gb300 as aim
    p1 = gen.generate(gen.WFA_150BP, 3000)
    p2 = gen.generate(gen.WFA_150BP, 3000, first=3000)
    # same shapes: every read 150 bp, targets of varying length -> pad both batches into fixed slots
    slot = 160
    def slots(p):
        buf = np.full(2 * len(p) * slot, ord("A"), np.uint8)
        for i in range(len(p)):
            r, t = p.read(i), p.target(i)
            buf[2 * i * slot:2 * i * slot + len(r)] = np.frombuffer(r, np.uint8)
            buf[(2 * i + 1) * slot:(2 * i + 1) * slot + len(t)] = np.frombuffer(t, np.uint8)
        return buf
    n = len(p1)
    ro = np.arange(n, dtype=np.int64) * 2 * slot; to = ro + slot
    buf, ro_d, to_d = aim.upload(slots(p1), ro, to)
    rl, tl = aim.upload(p1.read_len, p1.target_len)
    al = aim.Aligner(0, 1 << 30)
    out = al.outputs(n)
    plan = aim.aim_batch_plan(al.ctx, buf, buf, ro_d, to_d, rl, tl, slot, aim.penalties(4, 6, 2), 6, None,
                              out["scores"], None, None, out["cigar_lens"], out["flags"], autotune=False)
    aim.aim_batch_run(plan); torch.cuda.synchronize()
    a = out["scores"].cpu().numpy().copy()
    buf.copy_(torch.from_numpy(slots(p2)).cuda()); tl.copy_(torch.from_numpy(p2.target_len.view(np.int32)).cuda())
    aim.aim_batch_run(plan); torch.cuda.synchronize()
    b = out["scores"].cpu().numpy().copy()
    aim.aim_batch_destroy(plan); al.close()
    assert np.array_equal(a, device_results(p1, "wfa", AFF, 6)[0])
    assert np.array_equal(b, device_results(p2, "wfa", AFF, 6)[0])
