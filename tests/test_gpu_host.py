"""aim_align_batch_host: host buffers in, host buffers out, the transfers inside the call.  Results must equal the
device entry point's bit for bit, over several chunks with a short last one, for the batched wavefront path and
the plain DP path, with pinned and with pageable host arrays, on repeated calls (the context keeps its slots and
plans) and after a change of shape."""
import numpy as np
import pytest

import gen
import oracle
from devutil import assert_flat_same, device_flat, runs_capacity

pytestmark = pytest.mark.gpu

AFF = (0, 4, 6, 2)


def _host_call(aim, ctx, p, algo, pen, max_edits, cap, per_pair=None, band=-1, chunk=0, pinned=True, off=None):
    import torch
    n = len(p)

    def arr(a):
        if not pinned:
            return np.ascontiguousarray(a)
        t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True)
        out = t.numpy().view(a.dtype)
        out[...] = a
        return out

    def pinned_like(dtype, size):
        if not pinned:
            return np.zeros(size, dtype)
        tdt = {np.int32: torch.int32, np.uint8: torch.uint8, np.uint32: torch.int32, np.uint64: torch.int64}[dtype]
        a = torch.zeros(size, dtype=tdt, pin_memory=True).numpy()
        return a.view(dtype) if a.dtype != np.dtype(dtype) else a

    if off is None:
        off = np.zeros(n + 1, np.uint64); off[1:] = np.cumsum(cap)
    reads = arr(p.reads); targets = arr(p.targets)
    ro = arr(p.read_off.view(np.int64)).view(np.uint64); to = arr(p.target_off.view(np.int64)).view(np.uint64)
    rl = arr(p.read_len.view(np.int32)).view(np.uint32); tl = arr(p.target_len.view(np.int32)).view(np.uint32)
    coff = arr(off.view(np.int64)).view(np.uint64)
    me = arr(per_pair.astype(np.int32)) if per_pair is not None else None
    scores = pinned_like(np.int32, n); flags = pinned_like(np.uint8, n); lens = pinned_like(np.uint32, n)
    cig = pinned_like(np.uint32, int(off[-1]))
    ml = int(max(p.read_len.max(), p.target_len.max()))
    moved = aim.aim_align_batch_host(ctx, reads, targets, ro, to, rl, tl, ml, algo,
                                     aim.penalties(pen[1], pen[2], pen[3], band=band), max_edits, me, scores, cig,
                                     coff, lens, flags, chunk_pairs=chunk)
    return (scores.copy(), flags.copy(), lens.copy(), cig.copy(), off.astype(np.int64)), moved


def test_host_entry_point_equals_device_entry_point(oracle_lib, gen_lib):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim
    al = aim.Aligner(0, 2 << 30)
    w = gen.WFA_UNEVEN
    p = gen.generate(w, 50_003)
    me = gen.per_pair_max_edits(w, p)
    cap = runs_capacity(AFF, me)
    ref = device_flat(p, "wfa", AFF, int(me.max()), cap, per_pair=me, aligner=al)
    ref = (ref[0], ref[1], ref[2], ref[3], ref[4])
    orc_like = (ref[0], ref[1], ref[4], ref[3], ref[2])          # the comparator's (scores, flags, off, cigars, lens)
    # several chunks with a short last one; twice in a row (the second call replays the kept plans)
    for rep in range(2):
        got, moved = _host_call(aim, al.ctx, p, "wfa", AFF, int(me.max()), cap, per_pair=me, chunk=12_000)
        assert_flat_same(got, orc_like, what=f"host wfa, call {rep}")
        assert moved[0] >= p.reads.nbytes + p.targets.nbytes and moved[1] >= 9 * len(p)
    # pageable host arrays, one chunk
    got, _ = _host_call(aim, al.ctx, p, "wfa", AFF, int(me.max()), cap, per_pair=me, pinned=False)
    assert_flat_same(got, orc_like, what="host wfa, pageable")
    # another shape: banded Gotoh on 250 bp pairs (the plain path per chunk), against the oracle on a sample
    w3 = gen.GOTOH_WFA_250BP
    p3 = gen.generate(w3, 20_001)
    cap3 = runs_capacity(AFF, np.full(len(p3), 25))
    ref3 = device_flat(p3, "gotoh", AFF, 25, cap3, band=25, aligner=al)
    got3, _ = _host_call(aim, al.ctx, p3, "gotoh", AFF, 25, cap3, band=25, chunk=7_000)
    assert_flat_same(got3, (ref3[0], ref3[1], ref3[4], ref3[3], ref3[2]), what="host gotoh")
    sub = gen.generate(w3, 500)
    orc = oracle.align_batch(sub, AFF, np.full(500, oracle.limit_for(AFF, 25), np.int64), band=25,
                             cigar_cap=cap3[:500])
    assert_flat_same((got3[0][:500], got3[1][:500], got3[2][:500], got3[3][:int(orc[2][-1])], orc[2]), orc,
                     what="host gotoh vs oracle")
    al.close()


def test_host_slots_grow_for_later_chunks(oracle_lib, gen_lib):
    """The slots are sized from the first chunk; a later chunk with far longer sequences makes the call finish
    the earlier chunks, rebuild (and replan) its slots and go on: the results still equal the device entry
    point's, and a second call of the same shape reuses the grown slots.  A decreasing CIGAR offset in a later
    chunk is an argument error."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim
    al = aim.Aligner(0, 2 << 30)
    ps = gen.generate(gen.WFA_150BP, 6_000)
    pu = gen.generate(gen.WFA_UNEVEN, 9_001)
    p = gen.concat([ps, pu])
    me = np.concatenate([np.full(len(ps), 6, np.int32), gen.per_pair_max_edits(gen.WFA_UNEVEN, pu)])
    cap = runs_capacity(AFF, me)
    ref = device_flat(p, "wfa", AFF, int(me.max()), cap, per_pair=me, aligner=al)
    want = (ref[0], ref[1], ref[4], ref[3], ref[2])
    for rep in range(2):
        got, _ = _host_call(aim, al.ctx, p, "wfa", AFF, int(me.max()), cap, per_pair=me, chunk=3_000)
        assert_flat_same(got, want, what=f"host wfa, growing slots, call {rep}")
    refe = device_flat(p, "edit", (0, 1, 0, 1), 12, runs_capacity((0, 1, 0, 1), np.full(len(p), 12), unit=True),
                       aligner=al)
    gote, _ = _host_call(aim, al.ctx, p, "edit", (0, 1, 0, 1), 12,
                         runs_capacity((0, 1, 0, 1), np.full(len(p), 12), unit=True), chunk=3_000)
    assert_flat_same(gote, (refe[0], refe[1], refe[4], refe[3], refe[2]), what="host edit, growing slots")
    off = np.zeros(len(p) + 1, np.uint64); off[1:] = np.cumsum(cap)
    off[4_500] = off[4_499] - 1 if off[4_499] > 0 else 0   # decreasing entry inside the second chunk
    off[4_499] += 1
    with pytest.raises(aim.AimError):
        _host_call(aim, al.ctx, p, "wfa", AFF, int(me.max()), cap, per_pair=me, chunk=3_000, off=off)
    al.close()
