"""The client's cuckoo placement in parallel rounds on the device
(pepsi_params.client_cuckoo = 1), through pepsi_query: the placement equals
a plain Python restatement of the rounds (each unplaced item claims its
current candidate bin; the smallest claimant takes a free slot or evicts the
occupant of slot evictions mod gamma, which moves to its next candidate; the
other claimants move to theirs), is valid (every item in one of its three
candidate bins, at most gamma per bin), and the request's words equal the
oracle's encoding and encryption of that placement's table.  The evaluation
then decrypts to the hashed-domain brute force."""
import math

import numpy as np
import pytest

from cuckoo_rounds import rounds_reference
from gpu_helpers import T, torch_cuda

pytestmark = pytest.mark.gpu

PAPER = [55, 55, 54, 54]
DUMMY = (1 << 64) - 1


@pytest.mark.parametrize("gamma,blocks", [(1, 1), (2, 1), (1, 2)])
def test_device_cuckoo_rounds_valid_and_encrypted_as_the_oracle(gamma, blocks):
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    import paper_2310_14565_gb300 as pepsi

    torch_cuda()
    N, lb, h = 64, 10, 4
    bins = N * blocks
    logb = int(math.log2(bins))
    m = int(0.85 * gamma * bins)
    sets = make_sets(m, 3 * bins, 8, bits=32, seed_items=61 + gamma, seed_plant=62 + blocks)
    mu = max(6, oracle.simple_hash(0x5EED, lb, logb, sets.server, 1000)[2])
    gc = pepsi.Context(N=N, t=T, prime_bits=PAPER, h=h, lambda_bar=lb, mu=mu, hash_key=0x5EED, key_seed=3,
                       bins=bins, gamma=gamma, response_primes=1, client_cuckoo=1)
    oc = oracle.Ctx(N=N, t=T, prime_bits=PAPER, h=h, lambda_bar=lb, mu=mu, hash_key=0x5EED, bins=bins, gamma=gamma)
    s, rlk = oc.keygen(3)
    cts, where = gc.query(sets.client, 4)
    cts2, where2 = gc.query(sets.client, 4)
    assert np.array_equal(where, where2) and np.array_equal(cts, cts2)  # deterministic
    # the rounds, restated
    hashed = [oracle.hash_item(0x5EED, lb, logb, int(x)) for x in sets.client]
    ref = rounds_reference([b for _, b in hashed], gamma, bins)
    assert ref is not None and list(where) == ref
    # valid placement: one of the item's candidate bins, distinct slots
    assert len(set(int(w) for w in where)) == m
    for u, (_, b3) in enumerate(hashed):
        assert int(where[u]) // gamma in b3
    # the oracle's encoding and encryption of this placement's table
    table = np.full(bins * gamma, DUMMY, np.uint64)
    for u, (xl, _) in enumerate(hashed):
        table[where[u]] = xl
    cols = table.reshape(bins, gamma)
    pts = np.concatenate([oc.query_plaintexts(np.ascontiguousarray(cols[b * N:(b + 1) * N, i]))
                          for b in range(blocks) for i in range(gamma)])
    want = oc.encrypt(s, pts, 4).reshape(cts.shape)
    assert np.array_equal(cts, want)
    # the evaluation decrypts to the hashed-domain brute force
    sid = gc.server_load(sets.server)
    slots, budget = gc.decrypt(gc.eval(sid, cts))
    srv = {}
    for y in sets.server:
        yl, bb = oracle.hash_item(0x5EED, lb, logb, int(y))
        for b in bb:
            srv.setdefault(int(b), set()).add(yl)
    expect = np.zeros(bins * gamma, np.uint32)
    for u, (xl, _) in enumerate(hashed):
        expect[where[u]] = int(xl in srv.get(int(where[u]) // gamma, set()))
    assert budget > 0 and np.array_equal(slots, expect) and int(expect.sum()) >= 8


def test_device_cuckoo_fails_on_more_items_than_slots():
    from paper_2310_14565_gb300.workload import make_sets

    import paper_2310_14565_gb300 as pepsi

    torch_cuda()
    gc = pepsi.Context(N=64, t=T, prime_bits=PAPER, h=4, lambda_bar=10, mu=8, hash_key=0x5EED, client_cuckoo=1)
    sets = make_sets(65, 100, 2, bits=32, seed_items=71, seed_plant=72)
    with pytest.raises(pepsi.PepsiError) as err:
        gc.query(sets.client, 4)
    assert err.value.code == pepsi.E_CUCKOO_FAIL
    with pytest.raises(pepsi.PepsiError):
        pepsi.Context(N=64, t=T, prime_bits=PAPER, h=4, lambda_bar=10, mu=8, client_cuckoo=2)
