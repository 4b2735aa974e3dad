"""The continuous-batching engine (pepsi_engine_*), through the C ABI: every
request's result equals its solo pepsi_eval call word for word (and the
oracle's words), whatever else is in flight, for requests that arrive while
others run, join a lane's carousel at different layers, share the
multiply-accumulate with up to three others, and run on lanes of different
contexts (N, h, prime sets, rounding) at the same time."""
import math
import os

import numpy as np
import pytest

from gpu_helpers import T, pair, torch_cuda

pytestmark = pytest.mark.gpu

PAPER = [55, 55, 54, 54]
TOY = [36, 36, 37]
ALL = 0xFFFFFFFF


@pytest.fixture(autouse=True)
def _cuda():
    torch_cuda()


def _ctx(N, bits, h, lb, mu, chunk, **kw):
    os.environ["PEPSI_CHUNK"] = str(chunk)
    try:
        return pair(N, bits, h, lb, mu=mu, **kw)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)


def _sets(n, seed):
    from paper_2310_14565_gb300.workload import make_sets

    return make_sets(20, n, 4, bits=32, seed_items=seed, seed_plant=seed + 1)


def _mu(sets_list, lb, N):
    import oracle

    return max(oracle.simple_hash(0x5EED, lb, int(math.log2(N)), s.server, 100000)[2] for s in sets_list)


def _cases():
    """Two contexts: A (N = 64, four primes, h = 4, one rounding for all
    layers, one-prime response, value products in B) with two sets, one of
    them with values; B (N = 64, three primes, h = 2, per-layer rounding,
    plaintexts regenerated per chunk) with one set."""
    sA1, sA2, sB1 = _sets(90, 31), _sets(70, 33), _sets(80, 35)
    muA = max(9, _mu([sA1, sA2], 10, 64))
    ocA, gA, sA, rlkA = _ctx(64, PAPER, 4, 10, muA, 3, rescale_group=ALL, response_primes=1, server_values=1)
    valsA = (np.arange(len(sA1.server), dtype=np.uint64) * 7919 % 65536 + 1).astype(np.uint32)
    a1 = gA.server_load_values(sA1.server, valsA)
    a2 = gA.server_load(sA2.server)
    muB = max(7, _mu([sB1], 8, 64))
    ocB, gB, sB, rlkB = _ctx(64, TOY, 2, 8, muB, 2, resident_bytes=(1 << 64) - 1)
    b1 = gB.server_load(sB1.server)
    return dict(A=(ocA, gA, rlkA, sA1, sA2, a1, a2, valsA, muA), B=(ocB, gB, rlkB, sB1, b1, muB))


def _requests(g, sets, n, seed0):
    """n requests on a context: client sets with a few of the server's items."""
    out = []
    for i in range(n):
        cl = _sets(60, 100 + seed0 + i).client.copy()
        cl[:3] = sets.server[i:i + 3]
        out.append(g.query(cl, seed0 + i)[0])
    return out


def test_engine_words_equal_solo_calls_and_oracle():
    import oracle
    import paper_2310_14565_gb300 as pepsi

    c = _cases()
    ocA, gA, rlkA, sA1, sA2, a1, a2, valsA, muA = c["A"]
    ocB, gB, rlkB, sB1, b1, muB = c["B"]
    eng = pepsi.Engine([(gA, a1, 4), (gA, a2, 2), (gB, b1, 3)])
    reqA1 = _requests(gA, sA1, 6, 500)
    reqA2 = _requests(gA, sA2, 3, 600)
    reqB1 = _requests(gB, sB1, 5, 700)
    plan = ([(0, x, m, 10 + i) for i, (x, m) in enumerate(zip(reqA1, [0, 1, 2, 3, 2, 0]))] +
            [(1, x, i % 2, 20 + i) for i, x in enumerate(reqA2)] +
            [(2, x, i % 2, 30 + i) for i, x in enumerate(reqB1)])
    order = np.random.default_rng(7).permutation(len(plan))
    tickets = []
    for j, idx in enumerate(order):  # arrivals interleaved with scheduling passes
        lane, cts, mode, seed = plan[idx]
        t, out = eng.submit(lane, cts, mode=mode, mask_seed=seed)
        tickets.append((idx, t, out))
        for _ in range(j % 3):
            eng.pump()
    for idx, t, out in tickets:
        eng.wait(t)
    st = eng.stats()
    assert st["submitted"] == st["completed"] == len(plan) and st["bytes_in_use"] == 0
    _, TA1, VA1, _ = oracle.simple_hash_values(0x5EED, 10, 6, sA1.server, valsA, muA)
    _, TA2, _ = ocA.server_table(sA2.server)
    _, TB1, _ = ocB.server_table(sB1.server)
    ctxs = {0: (gA, a1), 1: (gA, a2), 2: (gB, b1)}
    for idx, t, out in tickets:
        lane, cts, mode, seed = plan[idx]
        g, sid = ctxs[lane]
        assert np.array_equal(out, g.eval(sid, cts, mode=mode, mask_seed=seed)), (lane, idx)
    for idx, t, out in tickets[:6]:  # a sample against the oracle
        lane, cts, mode, seed = plan[idx]
        if lane == 2:
            want = ocB.eval(rlkB, cts, TB1, mode=mode, mask_seed=seed)
        else:
            TT, V = (TA1, VA1) if lane == 0 else (TA2, None)
            want = ocA.mod_switch(ocA.eval(rlkA, cts, TT, mode=mode, mask_seed=seed, group=muA, V=V), 1)
        assert np.array_equal(out, want), (lane, idx)
    eng.close()


def test_engine_thread_device_buffers_and_budget():
    """The engine's own thread serves requests submitted from this thread,
    with device buffers; a budget that holds one request at a time still
    completes all of them, one after another, with the same words."""
    import paper_2310_14565_gb300 as pepsi

    torch = torch_cuda()
    c = _cases()
    ocA, gA, rlkA, sA1, sA2, a1, a2, valsA, muA = c["A"]
    reqs = _requests(gA, sA2, 6, 800)
    dev = [torch.from_numpy(x.view(np.int64).copy()).cuda() for x in reqs]
    outs = [torch.zeros(2 * 64, dtype=torch.int64, device="cuda") for _ in reqs]
    torch.cuda.synchronize()
    # one request's device state: the prepared request (split words and their 32-bit half sums,
    # 12 bytes per word), h' of a 3-layer chunk, the layer sum and the lazy run sum
    one = (gA.ell * 3 * gA.k * 64 + 3 * 2 * gA.k * 64 + 3 * gA.k * 64 + 3 * (gA.k + gA.kb) * 64) * 8
    for budget, slots in ((0, 4), (one, 4)):
        eng = pepsi.Engine([(gA, a2, slots)], hbm_budget=budget)
        eng.start()
        tk = [eng.submit(0, dev[i], out=outs[i], mode=i % 2, mask_seed=40 + i)[0] for i in range(len(reqs))]
        lat = [eng.wait(t) for t in tk]
        eng.stop()
        st = eng.stats()
        assert st["completed"] == len(reqs) and min(lat) > 0
        if budget:
            assert st["bytes_peak"] <= budget
        for i in range(len(reqs)):
            got = outs[i].cpu().numpy().view(np.uint64).reshape(2, 1, 64)
            assert np.array_equal(got, gA.eval(a2, reqs[i], mode=i % 2, mask_seed=40 + i)), (budget, i)
        eng.close()


def test_engine_rejects_unsupported_lanes():
    import paper_2310_14565_gb300 as pepsi

    sets = _sets(70, 41)
    mu = max(8, _mu([sets], 10, 64))
    _, g3, _, _ = _ctx(64, PAPER, 4, 10, mu, 3, rescale_group=3)  # runs of 3 layers depend on the start layer
    sid = g3.server_load(sets.server)
    with pytest.raises(pepsi.PepsiError):
        pepsi.Engine([(g3, sid, 2)])
    _, g1, _, _ = _ctx(64, PAPER, 4, 10, mu, 3)
    s1 = g1.server_load(sets.server)
    with pytest.raises(pepsi.PepsiError):
        pepsi.Engine([(g1, s1, 5)])  # more than four slots
    _, gb, _, _ = _ctx(64, PAPER, 4, 10, mu, 3, bins=128)
    sb = gb.server_load(sets.server)
    with pytest.raises(pepsi.PepsiError):
        pepsi.Engine([(gb, sb, 2)])  # two blocks of bins
    eng = pepsi.Engine([(g1, s1, 2)])
    with pytest.raises(pepsi.PepsiError):
        eng.submit(0, np.zeros((g1.ell, 2, g1.k, 64), np.uint64), mode=2)  # no values on this set
    eng.close()


def test_engine_captured_graph_replays_with_new_requests():
    """The batched form under one captured CUDA graph: requests on lanes of
    two contexts captured at once, launched, then the request buffers are
    refilled with other requests and the graph launched again; every output
    equals the solo call on the requests of that launch."""
    import paper_2310_14565_gb300 as pepsi

    torch = torch_cuda()
    c = _cases()
    ocA, gA, rlkA, sA1, sA2, a1, a2, valsA, muA = c["A"]
    ocB, gB, rlkB, sB1, b1, muB = c["B"]
    eng = pepsi.Engine([(gA, a2, 2), (gB, b1, 3)])
    first = _requests(gA, sA2, 3, 900) + _requests(gB, sB1, 4, 950)
    second = _requests(gA, sA2, 3, 1900) + _requests(gB, sB1, 4, 1950)
    lanes = [0] * 3 + [1] * 4
    ctxs = [(gA, a2)] * 3 + [(gB, b1)] * 4
    modes = [0, 1, 0, 1, 0, 1, 1]
    dev = [torch.from_numpy(x.view(np.int64).copy()).cuda() for x in first]
    outs = [torch.zeros(2 * g.response_primes * 64, dtype=torch.int64, device="cuda") for g, _ in ctxs]
    torch.cuda.synchronize()
    for i in range(len(dev)):
        eng.submit(lanes[i], dev[i], out=outs[i], mode=modes[i], mask_seed=60 + i)
    graph = eng.capture()
    for reqs in (first, second):
        for i, x in enumerate(reqs):
            dev[i].copy_(torch.from_numpy(x.view(np.int64)))
        torch.cuda.synchronize()
        graph.launch()
        for i, (g, sid) in enumerate(ctxs):
            got = outs[i].cpu().numpy().view(np.uint64).reshape(2, g.response_primes, 64)
            assert np.array_equal(got, g.eval(sid, reqs[i], mode=modes[i], mask_seed=60 + i)), i
    st = eng.stats()
    assert st["completed"] == len(dev)
    graph.close()
    eng.close()


def test_engine_failed_request_reports_its_status_and_others_complete():
    """A failure made on the host (the lane's next admission reports
    E_NOMEM instead of running): that request's wait returns the status, the
    engine's run returns it, and every other request, before and after it on
    the same lane and on another lane, completes with the solo call's words;
    the budget is given back."""
    import paper_2310_14565_gb300 as pepsi

    c = _cases()
    ocA, gA, rlkA, sA1, sA2, a1, a2, valsA, muA = c["A"]
    ocB, gB, rlkB, sB1, b1, muB = c["B"]
    eng = pepsi.Engine([(gA, a2, 2), (gB, b1, 2)])
    reqA = _requests(gA, sA2, 3, 1100)
    reqB = _requests(gB, sB1, 2, 1200)
    tA0, oA0 = eng.submit(0, reqA[0])
    eng.pump()  # admitted normally
    eng.fail_next(0, pepsi.E_NOMEM)
    tA1, oA1 = eng.submit(0, reqA[1], mode=1, mask_seed=3)
    tA2, oA2 = eng.submit(0, reqA[2])
    tB = [eng.submit(1, x) for x in reqB]
    with pytest.raises(pepsi.PepsiError) as err:
        eng.run()
    assert err.value.code == pepsi.E_NOMEM
    with pytest.raises(pepsi.PepsiError) as err:
        eng.wait(tA1)
    assert err.value.code == pepsi.E_NOMEM
    eng.wait(tA0)
    eng.wait(tA2)
    assert np.array_equal(oA0, gA.eval(a2, reqA[0])) and np.array_equal(oA2, gA.eval(a2, reqA[2]))
    for (t, o), x in zip(tB, reqB):
        eng.wait(t)
        assert np.array_equal(o, gB.eval(b1, x))
    st = eng.stats()
    assert st["completed"] == st["submitted"] == 5 and st["bytes_in_use"] == 0
    eng.close()
