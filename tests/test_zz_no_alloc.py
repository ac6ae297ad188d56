"""aim_wfa_align_static, the allocation-free WFA entry point, against aim_align_batch.

Callers that cannot allocate device memory (a plugin held to a fixed
device-memory budget by its host application, a loop that must not make a
call that can block on the device, a process whose footprint is fixed at
start-up) use aim_wfa_align_static, which runs the same wavefront kernel on a
fixed scratch array inside the library.  Two calls in a row, on different
batches, must give exactly what the context-based entry point gives: the
shared scratch keeps the previous call's contents, so the second call checks
that nothing leaks from one call into the next.  The second call runs on a
non-default stream, and the device's free memory and torch's allocation count
must be the same before and after it.  This file is collected last.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

AFF = (0, 4, 6, 2)


def _device_batch(aim, al, p, max_edits_per_pair=None):
    import torch
    n = len(p)
    wr = np.zeros(n, np.int64); wt = np.zeros(n, np.int64)
    wr[1:] = np.cumsum((p.read_len[:-1].astype(np.int64) + 31) // 32)
    wt[1:] = np.cumsum((p.target_len[:-1].astype(np.int64) + 31) // 32)
    nwr = int(wr[-1] + (int(p.read_len[-1]) + 31) // 32)
    nwt = int(wt[-1] + (int(p.target_len[-1]) + 31) // 32)
    cap = p.read_len.astype(np.int64) + p.target_len.astype(np.int64) + 1
    coff = np.zeros(n + 1, np.int64); coff[1:] = np.cumsum(cap)
    reads, targets, ro, to, rl, tl, wro, wto, coff_d = aim.upload(p.reads, p.targets, p.read_off, p.target_off,
                                                                  p.read_len, p.target_len, wr, wt, coff)
    pr = torch.zeros(nwr, dtype=torch.int64, device=rl.device)
    pt = torch.zeros(nwt, dtype=torch.int64, device=rl.device)
    aim.aim_pack_2bit(al.ctx, reads, ro, rl, pr, wro)
    aim.aim_pack_2bit(al.ctx, targets, to, tl, pt, wto)
    pp = aim.upload(max_edits_per_pair.astype(np.int32))[0] if max_edits_per_pair is not None else None
    return {"pr": pr, "pt": pt, "wro": wro, "wto": wto, "rl": rl, "tl": tl, "coff": coff_d, "pp": pp,
            "n": n, "ncig": int(coff[-1]), "max_len": int(max(p.read_len.max(), p.target_len.max()))}


def _outputs(b):
    import torch
    dev = b["rl"].device
    return {"scores": torch.full((b["n"],), -7, dtype=torch.int32, device=dev),
            "flags": torch.full((b["n"],), 255, dtype=torch.uint8, device=dev),
            "lens": torch.zeros(b["n"], dtype=torch.int32, device=dev),
            "cigars": torch.zeros(b["ncig"], dtype=torch.int32, device=dev)}


def test_static_scratch_entry_point_matches_context_entry_point():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim

    al = aim.Aligner(0, 1 << 30)     # the test itself may allocate: inputs, outputs, the reference call
    pen = aim.penalties(4, 6, 2)
    batches = [(gen.generate(gen.WFA_150BP, 3001), 6, None)]
    pu = gen.generate(gen.WFA_UNEVEN, 701)
    me = gen.per_pair_max_edits(gen.WFA_UNEVEN, pu)
    batches.append((pu, int(me.max()), me))
    side = torch.cuda.Stream()
    for call, (p, max_edits, per_pair) in enumerate(batches):       # two calls in a row
        b = _device_batch(aim, al, p, per_pair)
        ref, got = _outputs(b), _outputs(b)
        aim.aim_align_batch(al.ctx, b["pr"], b["pt"], b["wro"], b["wto"], b["rl"], b["tl"], b["max_len"], "wfa", pen,
                            max_edits, b["pp"], ref["scores"], ref["cigars"], b["coff"], ref["lens"], ref["flags"])
        torch.cuda.synchronize()
        free0, allocated0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        # the first call on the default stream, the second on another stream
        stream = None if call == 0 else side
        aim.aim_wfa_align_static(b["pr"], b["pt"], b["wro"], b["wto"], b["rl"], b["tl"], b["max_len"], pen,
                                 max_edits, b["pp"], got["scores"], got["cigars"], b["coff"], got["lens"],
                                 got["flags"], stream=stream)
        torch.cuda.synchronize()
        if call > 0:          # after the first call (module loaded, address looked up) nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == allocated0
        for k in ref:
            assert torch.equal(ref[k], got[k]), f"call {call}: {k} differs"
        assert int((ref["flags"] == 0).sum()) > 0

    # a request whose per-pair scratch exceeds the fixed array is refused with a clear status
    b = _device_batch(aim, al, gen.from_strings(["ACGT" * 8000], ["ACGT" * 8000]))
    out = _outputs(b)
    with pytest.raises(aim.AimError) as ei:
        aim.aim_wfa_align_static(b["pr"], b["pt"], b["wro"], b["wto"], b["rl"], b["tl"], b["max_len"], pen, -1, None,
                                 out["scores"], out["cigars"], b["coff"], out["lens"], out["flags"])
    assert ei.value.status == aim.AIM_ERR_NOMEM
    al.close()
