"""Client bins of gamma > 1 items (Section 4's client maximum bin load;
Algorithm 2 compares each client batch with every server layer), through the
C ABI against the oracle, word for word: the bucketed cuckoo table (bin of
every item), the request's gamma batches of ciphertexts, and one response
ciphertext per batch, with and without more bins than slots, indicator and
cardinality, both roundings.  Decryption gives the hashed-domain brute force
for every client item (more client items than bins)."""
import math

import numpy as np
import pytest

from gpu_helpers import T, pair, torch_cuda

pytestmark = pytest.mark.gpu

PAPER = [55, 55, 54, 54]
ALL = 0xFFFFFFFF


def _hashed_want(oracle, sets, where, bins, gamma, lb):
    logb = int(math.log2(bins))
    srv = {}
    for y in sets.server:
        yl, bb = oracle.hash_item(0x5EED, lb, logb, int(y))
        for b in bb:
            srv.setdefault(int(b), set()).add(yl)
    want = np.zeros(bins * gamma, np.uint32)
    for u, x in enumerate(sets.client):
        xl, _ = oracle.hash_item(0x5EED, lb, logb, int(x))
        want[where[u]] = int(xl in srv.get(int(where[u]) // gamma, set()))
    return want


@pytest.mark.parametrize("gamma,blocks,group", [(2, 1, ALL), (3, 1, 1), (2, 2, ALL)])
def test_gamma_batches_match_oracle(gamma, blocks, group):
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    torch_cuda()
    N, lb, h = 64, 10, 4
    bins = N * blocks
    m = int(0.8 * gamma * bins)  # more client items than bins
    sets = make_sets(m, 3 * bins, 8, bits=32, seed_items=80 + gamma, seed_plant=81 + blocks)
    logb = int(math.log2(bins))
    mu = max(6, oracle.simple_hash(0x5EED, lb, logb, sets.server, 1000)[2])
    oc = oracle.Ctx(N=N, t=T, prime_bits=PAPER, h=h, lambda_bar=lb, mu=mu, hash_key=0x5EED, bins=bins, gamma=gamma)
    _, gc, _, _ = pair(N, PAPER, h, lb, mu=mu, rescale_group=group, bins=bins, gamma=gamma, response_primes=1)
    s, rlk = oc.keygen(3)
    assert gc.gamma == gamma and gc.blocks == blocks
    rc, Ts, _ = oc.server_table(sets.server)
    assert rc == 0
    sid = gc.server_load(sets.server)
    cts, where = gc.query(sets.client, 4)
    rc, ocs, owhere = oc.query(s, sets.client, 4)
    assert rc == 0 and np.array_equal(where, owhere)
    assert cts.shape == ocs.shape and np.array_equal(cts, ocs)
    lead = ((blocks,) if blocks > 1 else ()) + (gamma,)
    flat = cts.reshape((blocks * gamma,) + cts.shape[-4:])
    for mode, seed in ((0, 0), (1, 7)):
        out = gc.eval(sid, cts, mode=mode, mask_seed=seed)
        assert out.shape == lead + (2, 1, N)
        got = out.reshape(blocks * gamma, 2, 1, N)
        for r in range(blocks * gamma):
            b = r // gamma
            G = mu if group == ALL else 1
            want = oc.mod_switch(oc.eval(rlk, flat[r], Ts[:, b * N:(b + 1) * N], mode=mode, mask_seed=seed + r,
                                         group=G), 1)
            assert np.array_equal(got[r], want), (mode, r)
        slots, budget = gc.decrypt(out)
        assert budget > 0 and slots.shape == (bins * gamma,)
        want = _hashed_want(oracle, sets, where, bins, gamma, lb)
        if mode == 0:
            assert np.array_equal(slots, want) and int(want.sum()) >= 8
        else:
            assert int(slots.astype(np.int64).sum()) % T == int(want.sum())
    # the batch form: two requests, the same words as single calls
    cts2, _ = gc.query(sets.client[::-1].copy(), 9)
    outs = gc.eval_batch([sid, sid], [cts, cts2], [0, 1], [0, 3])
    assert np.array_equal(outs[0], gc.eval(sid, cts))
    assert np.array_equal(outs[1], gc.eval(sid, cts2, mode=1, mask_seed=3))


def test_gamma_one_is_the_one_slot_request():
    """gamma = 1 (the paper's cuckoo hashing) keeps the request and response
    shapes and words of a context without the parameter."""
    from paper_2310_14565_gb300.workload import make_sets

    import paper_2310_14565_gb300 as pepsi

    torch_cuda()
    sets = make_sets(40, 150, 5, bits=32, seed_items=91, seed_plant=92)
    a = pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=24, hash_key=0x5EED, key_seed=3)
    b = pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=24, hash_key=0x5EED, key_seed=3, gamma=1)
    ca, wa = a.query(sets.client, 4)
    cb, wb = b.query(sets.client, 4)
    assert ca.shape == cb.shape == (a.ell, 2, 4, 64) and np.array_equal(ca, cb) and np.array_equal(wa, wb)
    sa, sb = a.server_load(sets.server), b.server_load(sets.server)
    assert np.array_equal(a.eval(sa, ca), b.eval(sb, cb))
    with pytest.raises(pepsi.PepsiError):
        pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=12, gamma=17)


def test_engine_serves_each_batch_of_a_gamma_request():
    """An engine lane over a context with gamma = 2 serves each client batch
    of a request as its own request: batch i with mask seed s + i gives the
    words of Context.eval on the whole request (indicator and cardinality)."""
    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300.workload import make_sets

    torch_cuda()
    gamma, N = 2, 64
    sets = make_sets(80, 200, 6, bits=32, seed_items=95, seed_plant=96)
    ctx = pepsi.Context(N=N, prime_bits=PAPER, h=4, lambda_bar=10, mu=24, hash_key=0x5EED, key_seed=3, gamma=gamma,
                        rescale_group=pepsi.RESCALE_ALL, response_primes=1)
    sid = ctx.server_load(sets.server)
    cts, _ = ctx.query(sets.client, 4)
    assert cts.shape[0] == gamma
    eng = pepsi.Engine([(ctx, sid, 4)])
    for mode, seed in ((0, 0), (1, 11)):
        want = ctx.eval(sid, cts, mode=mode, mask_seed=seed)
        tickets = [eng.submit(0, np.ascontiguousarray(cts[i]), mode=mode, mask_seed=seed + i) for i in range(gamma)]
        eng.run()
        for i, (t, out) in enumerate(tickets):
            eng.wait(t)
            assert np.array_equal(out, want[i]), (mode, i)
    eng.close()

