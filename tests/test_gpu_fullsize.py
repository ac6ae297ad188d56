"""Parity at the workloads' full sizes: every pair of the 150 bp and 250 bp workloads, 100,000 pairs of the uneven
workload through the batched form, and a sample of the serving workload's shape (100-10,000 bp, at least 200 pairs
of 5 kbp or more) through the serving loop, each compared with the oracle element by element: scores, flags, run
counts and every CIGAR run."""
import numpy as np
import pytest

import gen
import oracle
from devutil import assert_flat_same, device_flat, limits, runs_capacity

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


def test_wfa_150bp_every_pair(aligner, oracle_lib, gen_lib):
    """All 1,000,000 pairs of the 150 bp workload (4 % edits, 10 % unrelated, threshold 6 edits)."""
    w = gen.WFA_150BP
    p = gen.generate(w)
    assert len(p) == 1_000_000
    cap = runs_capacity(AFF, np.full(len(p), 6))
    orc = oracle.align_batch(p, AFF, limits(w, p), cigar_cap=cap)
    dev = device_flat(p, "wfa", AFF, 6, cap, aligner=aligner)
    assert_flat_same(dev, orc, what="wfa 150bp, all 1M pairs")
    rej = (orc[1] & oracle.F_REJECTED) > 0
    assert (rej <= p.unrelated.astype(bool)).all() and rej.sum() > 90_000


def test_gotoh_and_wfa_250bp_band25_every_pair(aligner, oracle_lib, gen_lib):
    """All 1,000,000 pairs of the 250 bp workload (10 % edits, band 25, threshold 25 edits), banded Gotoh DP and
    banded WFA, each against the banded full-matrix oracle."""
    w = gen.GOTOH_WFA_250BP
    p = gen.generate(w)
    assert len(p) == 1_000_000
    cap = runs_capacity(AFF, np.full(len(p), 25))
    orc = oracle.align_batch(p, AFF, limits(w, p), band=25, cigar_cap=cap)
    for algo in ("gotoh", "wfa"):
        dev = device_flat(p, algo, AFF, 25, cap, band=25, aligner=aligner)
        assert_flat_same(dev, orc, what=f"{algo} 250bp band 25, all 1M pairs")


def test_uneven_batched_100k_pairs(oracle_lib, gen_lib):
    """The first 100,000 pairs of the uneven workload (100-1000 bp, 1-10 % edits, thresholds 10 % of the length)
    through the batched form (planned, autotuned, replayed as a CUDA graph), against the oracle."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim
    w = gen.WFA_UNEVEN
    p = gen.generate(w, 100_000)
    me = gen.per_pair_max_edits(w, p)
    cap = runs_capacity(AFF, me)
    orc = oracle.align_batch(p, AFF, limits(w, p), cigar_cap=cap)
    n = len(p)
    off = np.zeros(n + 1, np.int64); off[1:] = np.cumsum(cap)
    reads, targets, ro, to, rl, tl, coff, pp = aim.upload(p.reads, p.targets, p.read_off, p.target_off, p.read_len,
                                                          p.target_len, off, me.astype(np.int32))
    al = aim.Aligner(0, 1 << 30)
    dev = rl.device
    scores = torch.full((n,), -7, dtype=torch.int32, device=dev)
    flags = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    lens = torch.zeros(n, dtype=torch.int32, device=dev)
    cig = torch.zeros(int(off[-1]), dtype=torch.int32, device=dev)
    ml = int(max(p.read_len.max(), p.target_len.max()))      # targets can outgrow their 1000 bp reads
    plan = aim.aim_batch_plan(al.ctx, reads, targets, ro, to, rl, tl, ml, aim.penalties(4, 6, 2), int(me.max()),
                              pp, scores, cig, coff, lens, flags, autotune=True)
    try:
        for _ in range(2):                 # two replays of the same plan
            scores.fill_(-7); flags.fill_(255); lens.zero_(); cig.zero_()
            aim.aim_batch_run(plan)
            torch.cuda.synchronize()
            got = (scores.cpu().numpy(), flags.cpu().numpy(), lens.cpu().numpy().view(np.uint32),
                   cig.cpu().numpy().view(np.uint32), off)
            assert_flat_same(got, orc, what="uneven batched, 100k pairs")
    finally:
        aim.aim_batch_destroy(plan)
        al.close()


def test_serving_shape_long_pairs(oracle_lib, gen_lib):
    """1,600 pairs of the serving workload's shape (reads log-uniform over 100-10,000 bp, 1-10 % edits,
    thresholds 10 % of the length; at least 200 of them 5 kbp or longer) submitted to the serving loop as requests
    of log-uniform sizes, all in flight together; every result against the row-block oracle, canonical CIGARs
    included."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim
    w = gen.SERVE_LONG
    p = gen.generate(w, 1_600)
    assert (p.read_len >= 5000).sum() >= 200
    me = gen.per_pair_max_edits(w, p)
    cap = runs_capacity(AFF, me)
    orc = oracle.align_batch(p, AFF, limits(w, p), cigar_cap=cap, rows_per_block=0)
    rng = np.random.default_rng(23)
    ctx = aim.aim_create(0, 64 << 20)
    srv = aim.aim_server_create(ctx, aim.penalties(4, 6, 2), 24 << 30, 1 << 30)
    subs, at = [], 0
    while at < len(p):
        k = min(int(np.floor(np.exp(rng.uniform(0, np.log(400))))), len(p) - at)
        idx = np.arange(at, at + k)
        at += k
        q = gen.concat([gen.from_strings([p.read(i)], [p.target(i)]) for i in idx])
        c = cap[idx]
        qoff = np.zeros(k + 1, np.uint64); qoff[1:] = np.cumsum(c)
        out = (np.full(k, -7, np.int32), np.full(k, 255, np.uint8), np.zeros(k, np.uint32),
               np.zeros(int(qoff[-1]), np.uint32), qoff)
        t, keep = aim.aim_server_submit(srv, q.reads, q.targets, q.read_off, q.target_off, q.read_len, q.target_len,
                                        me[idx].astype(np.int32), out[0], out[1], out[2], out[3], qoff)
        subs.append((t, keep, idx, out))
    for t, _, _, _ in subs:
        aim.aim_server_wait(srv, t)
    st = aim.aim_server_stats(srv)
    aim.aim_server_destroy(srv)
    aim.aim_destroy(ctx)
    assert st["failed"] == 0 and st["completed"] == len(subs)
    s = np.concatenate([o[0] for _, _, _, o in subs]); f = np.concatenate([o[1] for _, _, _, o in subs])
    ln = np.concatenate([o[2] for _, _, _, o in subs]); cg = np.concatenate([o[3] for _, _, _, o in subs])
    off = np.zeros(len(p) + 1, np.int64); off[1:] = np.cumsum(cap)
    assert_flat_same((s, f, ln, cg, off), orc, what="serving shape, 1,600 pairs")
    assert ((f == 0) & (p.read_len >= 5000)).sum() >= 150     # the long pairs are mostly accepted, CIGARs compared
