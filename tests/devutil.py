"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
bring results back as numpy; run the oracle on the same seeded pairs."""
from __future__ import annotations

import numpy as np

import gen
import oracle


def limits(w: gen.Workload, p: gen.Pairs) -> np.ndarray:
    unit = w.algo == "edit"
    return np.array([oracle.limit_for(w.penalties, int(k), unit=unit) for k in gen.per_pair_max_edits(w, p)],
                    np.int64)


def cigar_capacity(p: gen.Pairs) -> np.ndarray:
    return (p.read_len.astype(np.int64) + p.target_len.astype(np.int64) + 1)


def oracle_results(p: gen.Pairs, penalties, lim: np.ndarray, band: int = -1):
    s, f, off, cig, lens = oracle.align_batch(p, penalties, lim, band=band)
    runs = [cig[off[i]:off[i] + lens[i]].astype(np.uint32) for i in range(len(p))]
    return s, f, runs


def device_results(p: gen.Pairs, algo: str, penalties, max_edits: int, per_pair: np.ndarray | None = None,
                   band: int = -1, max_score: int = -1, path: str = "ascii", max_length: int | None = None,
                   cigar_cap: np.ndarray | None = None, workspace: int = 0, aligner=None):
    import torch
    import paper_2208_01243_gb300 as aim
    n = len(p)
    ml = int(max_length if max_length is not None else max(int(p.read_len.max(initial=0)),
                                                          int(p.target_len.max(initial=0)), 1))
    pen = aim.penalties(penalties[1], penalties[2], penalties[3], max_score=max_score, band=band)
    own = aligner is None
    al = aligner or aim.Aligner(0, workspace)
    cap = cigar_cap if cigar_cap is not None else cigar_capacity(p)
    off = np.zeros(n + 1, np.int64); off[1:] = np.cumsum(cap)
    (rl, tl, ro, to, reads, targets, coff) = aim.upload(p.read_len, p.target_len, p.read_off, p.target_off,
                                                        p.reads if len(p.reads) else np.zeros(1, np.uint8),
                                                        p.targets if len(p.targets) else np.zeros(1, np.uint8), off)
    dev = rl.device
    scores = torch.full((n,), -7, dtype=torch.int32, device=dev)
    flags = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    lens = torch.zeros(n, dtype=torch.int32, device=dev)
    cig = torch.zeros(max(int(off[-1]), 1), dtype=torch.int32, device=dev)
    pp = aim.upload(per_pair.astype(np.int32))[0] if per_pair is not None else None
    if path == "ascii":
        aim.aim_align_batch_ascii(al.ctx, reads, targets, ro, to, rl, tl, ml, algo, pen, max_edits, pp, scores, cig,
                                  coff, lens, flags)
    else:
        wr = np.zeros(n, np.int64); wt = np.zeros(n, np.int64)
        if n:
            wr[1:] = np.cumsum((p.read_len[:-1].astype(np.int64) + 31) // 32)
            wt[1:] = np.cumsum((p.target_len[:-1].astype(np.int64) + 31) // 32)
        nwr = int(wr[-1] + (int(p.read_len[-1]) + 31) // 32) if n else 0
        nwt = int(wt[-1] + (int(p.target_len[-1]) + 31) // 32) if n else 0
        pr = torch.zeros(max(nwr, 1), dtype=torch.int64, device=dev)
        pt = torch.zeros(max(nwt, 1), dtype=torch.int64, device=dev)
        wro, wto = aim.upload(wr, wt)
        aim.aim_pack_2bit(al.ctx, reads, ro, rl, pr, wro)
        aim.aim_pack_2bit(al.ctx, targets, to, tl, pt, wto)
        aim.aim_align_batch(al.ctx, pr, pt, wro, wto, rl, tl, ml, algo, pen, max_edits, pp, scores, cig, coff, lens,
                            flags)
    torch.cuda.synchronize()
    s = scores.cpu().numpy(); f = flags.cpu().numpy(); ln = lens.cpu().numpy().view(np.uint32)
    cg = cig.cpu().numpy().view(np.uint32)
    runs = [cg[off[i]:off[i] + min(int(ln[i]), int(cap[i]))] for i in range(n)]
    if own:
        al.close()
    return s, f, runs, ln


def assert_same(dev, orc, idx=None, what=""):
    ds, df, druns = dev[0], dev[1], dev[2]
    os_, of, oruns = orc
    idx = range(len(os_)) if idx is None else idx
    bad = []
    for j, i in enumerate(idx):
        ok = (int(ds[i]) == int(os_[j]) and int(df[i]) == int(of[j])
              and np.array_equal(np.asarray(druns[i], np.uint32), np.asarray(oruns[j], np.uint32)))
        if not ok:
            bad.append(i)
    if bad:
        i = bad[0]
        j = list(idx).index(i)
        raise AssertionError(f"{what}: {len(bad)} pairs differ; first pair {i}: device score {ds[i]} flags {df[i]} "
                             f"runs {list(druns[i])[:12]} vs oracle score {os_[j]} flags {of[j]} "
                             f"runs {list(oruns[j])[:12]}")


def runs_capacity(penalties, max_edits: np.ndarray, unit: bool = False) -> np.ndarray:
    """CIGAR runs an accepted pair can need: every edit run costs at least min(x, o+e), so a pair under the limit
    L = max_edits * max(x, o+e) has at most 2 * (L // min(x, o+e)) + 1 runs (unit costs: 2 * max_edits + 1)."""
    me = np.asarray(max_edits, np.int64)
    if unit:
        return 2 * me + 1
    _, x, o, e = penalties
    return 2 * ((me * max(x, o + e)) // min(x, o + e)) + 1


def device_flat(p: gen.Pairs, algo: str, penalties, max_edits: int, cap: np.ndarray, per_pair=None, band: int = -1,
                aligner=None):
    """The CUDA path over all pairs with one flat CIGAR array (pair i's runs at off[i], capacity cap[i]) ->
    (scores, flags, lens, cigars, off), zero past each pair's runs."""
    import torch
    import paper_2208_01243_gb300 as aim
    n = len(p)
    ml = int(max(int(p.read_len.max(initial=0)), int(p.target_len.max(initial=0)), 1))
    off = np.zeros(n + 1, np.int64); off[1:] = np.cumsum(cap)
    reads, targets, ro, to, rl, tl, coff = aim.upload(p.reads, p.targets, p.read_off, p.target_off, p.read_len,
                                                      p.target_len, off)
    dev = rl.device
    scores = torch.full((n,), -7, dtype=torch.int32, device=dev)
    flags = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    lens = torch.zeros(n, dtype=torch.int32, device=dev)
    cig = torch.zeros(max(int(off[-1]), 1), dtype=torch.int32, device=dev)
    pp = aim.upload(per_pair.astype(np.int32))[0] if per_pair is not None else None
    aim.aim_align_batch_ascii(aligner.ctx, reads, targets, ro, to, rl, tl, ml, algo,
                              aim.penalties(penalties[1], penalties[2], penalties[3], band=band), max_edits, pp,
                              scores, cig, coff, lens, flags)
    torch.cuda.synchronize()
    return (scores.cpu().numpy(), flags.cpu().numpy(), lens.cpu().numpy().view(np.uint32),
            cig.cpu().numpy().view(np.uint32)[:int(off[-1])], off)


def assert_flat_same(dev, orc, what=""):
    """Element by element: scores, flags, run counts and every CIGAR run (both sides zero past each pair's runs)."""
    ds, df, dl, dc, doff = dev
    os_, of, ooff, oc, ol = orc
    assert np.array_equal(np.asarray(doff, np.int64), np.asarray(ooff, np.int64)), f"{what}: CIGAR offsets differ"
    bad = np.nonzero((ds != os_) | (df != of) | (dl != ol))[0]
    if len(bad) == 0 and not np.array_equal(dc, oc):
        pos = int(np.nonzero(dc != oc)[0][0])
        bad = np.array([int(np.searchsorted(np.asarray(ooff, np.int64), pos, side="right") - 1)])
    if len(bad):
        i = int(bad[0])
        a, b = int(ooff[i]), int(ooff[i + 1])
        raise AssertionError(f"{what}: {len(bad)} pair(s) differ; first pair {i}: device ({ds[i]}, {df[i]}, "
                             f"{dl[i]} runs {list(dc[a:a + 8])}) oracle ({os_[i]}, {of[i]}, {ol[i]} runs "
                             f"{list(oc[a:a + 8])})")
