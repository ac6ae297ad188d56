"""Serving loop: each request's result is the same alone and in a mix that contends for the memory budget."""
import numpy as np
import pytest

import gen
import oracle
from devutil import device_results

pytestmark = pytest.mark.gpu

AFF = (0, 4, 6, 2)
MIXED = gen.Workload("serve_test_100_2000bp_1_10pct", 5, 0, 100, 2000, 0.01, 0.10, 0.0, "wfa", AFF, None,
                     max_edits_frac=0.10)


def _requests(n_req=40, seed=11):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(0, np.log(300), n_req))).astype(int)
    pool = gen.generate(MIXED, int(sizes.sum()))
    me = gen.per_pair_max_edits(MIXED, pool)
    reqs, at = [], 0
    for k in sizes:
        idx = np.arange(at, at + k)
        at += k
        reqs.append((idx, me[idx]))
    return pool, reqs


def _submit(aim, srv, pool, idx, me):
    p = gen.concat([gen.from_strings([pool.read(i)], [pool.target(i)]) for i in idx])
    n = len(p)
    cap = p.read_len.astype(np.int64) + p.target_len.astype(np.int64) + 1
    coff = np.zeros(n + 1, np.uint64); coff[1:] = np.cumsum(cap)
    out = {"scores": np.full(n, -7, np.int32), "flags": np.full(n, 255, np.uint8), "lens": np.zeros(n, np.uint32),
           "cigars": np.zeros(int(coff[-1]), np.uint32), "coff": coff, "pairs": p, "me": me}
    t, keep = aim.aim_server_submit(srv, p.reads, p.targets, p.read_off, p.target_off, p.read_len, p.target_len,
                                    me.astype(np.int32), out["scores"], out["flags"], out["lens"], out["cigars"], coff)
    out["keep"] = keep
    return t, out


def _runs(o):
    return [o["cigars"][o["coff"][i]:o["coff"][i] + o["lens"][i]] for i in range(len(o["scores"]))]


def test_results_same_alone_and_in_the_mix(oracle_lib, gen_lib):
    import __graft_entry__
    __graft_entry__.build()
    import paper_2208_01243_gb300 as aim
    pool, reqs = _requests()
    ctx = aim.aim_create(0, 64 << 20)
    pen = aim.penalties(4, 6, 2)
    # in the mix: everything submitted at once against a small wavefront budget, so requests queue and overlap
    srv = aim.aim_server_create(ctx, pen, 96 << 20, 256 << 20)
    subs = [_submit(aim, srv, pool, idx, me) for idx, me in reqs]
    lat = [aim.aim_server_wait(srv, t) for t, _ in subs]
    st = aim.aim_server_stats(srv)
    aim.aim_server_destroy(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0 and all(x > 0 for x in lat)
    # alone: one request at a time on a fresh server
    srv = aim.aim_server_create(ctx, pen, 96 << 20, 256 << 20)
    for (idx, me), (_, mixed) in zip(reqs, subs):
        t, alone = _submit(aim, srv, pool, idx, me)
        aim.aim_server_wait(srv, t)
        assert np.array_equal(alone["scores"], mixed["scores"]) and np.array_equal(alone["flags"], mixed["flags"])
        assert all(np.array_equal(a, b) for a, b in zip(_runs(alone), _runs(mixed)))
    aim.aim_server_destroy(srv)
    aim.aim_destroy(ctx)
    # and the same as the plain batch entry point, and the oracle on a sample
    for k in (0, len(reqs) // 2, len(reqs) - 1):
        o = subs[k][1]
        plain = device_results(o["pairs"], "wfa", AFF, int(o["me"].max()), per_pair=o["me"])
        assert np.array_equal(plain[0], o["scores"]) and np.array_equal(plain[1], o["flags"])
        assert all(np.array_equal(a, b) for a, b in zip(plain[2], _runs(o)))
        j = int(np.argmax(o["pairs"].read_len))
        s, f, runs = oracle.align(o["pairs"].read(j), o["pairs"].target(j), AFF,
                                  limit=oracle.limit_for(AFF, int(o["me"][j])))
        assert (s, f) == (o["scores"][j], o["flags"][j]) and list(runs) == list(_runs(o)[j])


def test_request_larger_than_the_budget_is_refused(gen_lib):
    import paper_2208_01243_gb300 as aim
    ctx = aim.aim_create(0, 64 << 20)
    srv = aim.aim_server_create(ctx, aim.penalties(4, 6, 2), 1 << 20, 64 << 20)
    p = gen.generate(gen.SERVE_LONG, 200)
    i = int(np.argmax(p.read_len))
    q = gen.from_strings([p.read(i)], [p.target(i)])
    out_s, out_f = np.zeros(1, np.int32), np.zeros(1, np.uint8)
    with pytest.raises(aim.AimError) as ei:
        aim.aim_server_submit(srv, q.reads, q.targets, q.read_off, q.target_off, q.read_len, q.target_len,
                              np.array([int(np.ceil(0.1 * q.read_len[0]))], np.int32), out_s, out_f)
    assert ei.value.status == aim.AIM_ERR_NOMEM
    aim.aim_server_destroy(srv)
    aim.aim_destroy(ctx)


def _same_as_plain(o):
    plain = device_results(o["pairs"], "wfa", AFF, int(o["me"].max()), per_pair=o["me"])
    assert np.array_equal(plain[0], o["scores"]) and np.array_equal(plain[1], o["flags"])
    assert all(np.array_equal(a, b) for a, b in zip(plain[2], _runs(o)))


def test_pause_cancel_and_an_injected_launch_failure(gen_lib):
    """Host-side failure paths: a paused server admits nothing; a queued request is cancelled and its outputs stay
    untouched; a request made to fail at launch (injected on the host, no GPU fault) completes with AIM_ERR_CUDA
    while the requests around it, and a later one, give the plain entry point's results."""
    import time
    import paper_2208_01243_gb300 as aim
    pool, reqs = _requests(n_req=6, seed=12)
    ctx = aim.aim_create(0, 64 << 20)
    srv = aim.aim_server_create(ctx, aim.penalties(4, 6, 2), 96 << 20, 256 << 20)
    aim.aim_server_pause(srv, True)
    subs = [_submit(aim, srv, pool, idx, me) for idx, me in reqs[:4]]
    time.sleep(0.05)
    st = aim.aim_server_stats(srv)
    assert (st["queued"], st["running"], st["completed"]) == (4, 0, 0)
    t1, o1 = subs[1]
    assert aim.aim_server_cancel(srv, t1)
    with pytest.raises(aim.AimError) as ei:
        aim.aim_server_wait(srv, t1)
    assert ei.value.status == aim.AIM_ERR_CANCELLED
    assert (o1["scores"] == -7).all() and (o1["flags"] == 255).all() and not o1["lens"].any()
    with pytest.raises(aim.AimError) as ei:   # the ticket is released
        aim.aim_server_cancel(srv, t1)
    assert ei.value.status == aim.AIM_ERR_ARG
    # admission order from here: requests 0, 2, 3; the second of them fails at launch
    aim.aim_server_inject_failure(srv, 2)
    aim.aim_server_pause(srv, False)
    aim.aim_server_wait(srv, subs[0][0])
    with pytest.raises(aim.AimError) as ei:
        aim.aim_server_wait(srv, subs[2][0])
    assert ei.value.status == aim.AIM_ERR_CUDA
    aim.aim_server_wait(srv, subs[3][0])
    _same_as_plain(subs[0][1])
    _same_as_plain(subs[3][1])
    # the server carries on; an admitted request cannot be cancelled
    t4, o4 = _submit(aim, srv, pool, *reqs[4])
    for _ in range(2000):
        if aim.aim_server_stats(srv)["completed"] == 5:
            break
        time.sleep(0.005)
    assert not aim.aim_server_cancel(srv, t4)
    aim.aim_server_wait(srv, t4)
    _same_as_plain(o4)
    st = aim.aim_server_stats(srv)
    assert (st["submitted"], st["completed"], st["failed"], st["queued"], st["running"]) == (5, 5, 2, 0, 0)
    aim.aim_server_destroy(srv)
    aim.aim_destroy(ctx)


def test_device_allocation_failures_leave_the_device_usable(gen_lib):
    """Budgets twice the device's memory: the allocation fails, the call returns AIM_ERR_NOMEM, and work runs
    afterwards."""
    import torch
    import paper_2208_01243_gb300 as aim
    too_much = 2 * torch.cuda.mem_get_info(0)[1]
    with pytest.raises(aim.AimError) as ei:
        aim.aim_create(0, too_much)
    assert ei.value.status == aim.AIM_ERR_NOMEM
    ctx = aim.aim_create(0, 64 << 20)
    with pytest.raises(aim.AimError) as ei:
        aim.aim_server_create(ctx, aim.penalties(4, 6, 2), too_much, 64 << 20)
    assert ei.value.status == aim.AIM_ERR_NOMEM
    pool, reqs = _requests(n_req=1, seed=13)
    srv = aim.aim_server_create(ctx, aim.penalties(4, 6, 2), 96 << 20, 256 << 20)
    t, o = _submit(aim, srv, pool, *reqs[0])
    aim.aim_server_wait(srv, t)
    aim.aim_server_destroy(srv)
    aim.aim_destroy(ctx)
    _same_as_plain(o)
