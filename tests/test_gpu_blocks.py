"""More bins than slots (pepsi_params.bins = B * N, Section 4's ceil(b/N)
ciphertexts per code bit): the request, the server table and plaintexts,
the per-block responses and the batch path against the oracle, word for
word; the blocks' slots together decrypt to the hashed-domain
intersection over all b bins."""
import math
import os

import numpy as np
import pytest

from gpu_helpers import T, hashed_indicator, torch_cuda

pytestmark = pytest.mark.gpu

PAPER = [55, 55, 54, 54]
ALL = 0xFFFFFFFF


@pytest.fixture(autouse=True)
def _cuda():
    torch_cuda()


def _case(B=4, N=64, group=0, values=False, response_primes=0, chunk=3):
    import oracle
    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300.workload import make_sets

    lb = 10
    bins = B * N
    sets = make_sets(150, 300, 9, bits=32, seed_items=71, seed_plant=72)
    vals = np.random.default_rng(5).integers(1, T, size=300).astype(np.uint32)
    mu = max(5, oracle.simple_hash(0x5EED, lb, int(math.log2(bins)), sets.server, 1000)[2])
    oc = oracle.Ctx(N=N, t=T, prime_bits=PAPER, h=4, lambda_bar=lb, mu=mu, hash_key=0x5EED, bins=bins)
    os.environ["PEPSI_CHUNK"] = str(chunk)
    try:
        gc = pepsi.Context(N=N, prime_bits=PAPER, h=4, lambda_bar=lb, mu=mu, hash_key=0x5EED, key_seed=3,
                           rescale_group=group, server_values=1, response_primes=response_primes, bins=bins)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    s, rlk = oc.keygen(3)
    if values:
        sid = gc.server_load_values(sets.server, vals)
        rc, Ts, V, _ = oc.server_table_values(sets.server, vals)
    else:
        sid = gc.server_load(sets.server)
        rc, Ts, _ = oc.server_table(sets.server)
        V = None
    assert rc == 0
    cts, where = gc.query(sets.client, 4)
    return oc, gc, s, rlk, sets, sid, Ts, V, cts, where, mu


def test_blocks_request_and_tables_match_oracle():
    oc, gc, s, rlk, sets, sid, Ts, V, cts, where, mu = _case(values=True)
    assert gc.bins == 256 and gc.blocks == 4
    rc, ocs, owhere = oc.query(s, sets.client, 4)
    assert rc == 0 and np.array_equal(where, owhere)
    assert cts.shape == (4, gc.ell, 2, 4, 64) and np.array_equal(cts, ocs)
    assert np.array_equal(gc.server_table(sid, mu), Ts)
    assert np.array_equal(gc.server_values(sid, mu), V)
    P = gc.server_plaintexts(sid, 1, 2)
    assert P.shape == (4, 2, gc.ell, 4, 64)
    for b in (0, 3):
        for j in (0, gc.ell - 1):
            assert np.array_equal(P[b, 1, j], oc.server_plaintext(Ts[:, b * 64:(b + 1) * 64], 2, j))


@pytest.mark.parametrize("group", [0, ALL])
def test_blocks_eval_all_modes_match_oracle(group):
    oc, gc, s, rlk, sets, sid, Ts, V, cts, where, mu = _case(values=True, group=group)
    og = mu if group == ALL else 1
    hashed = hashed_indicator(sets.client, sets.server, where, 256, 10)
    for mode in (0, 1, 2, 3):
        got = gc.eval(sid, cts, mode=mode, mask_seed=11)
        assert got.shape == (4, 2, 4, 64)
        for b in range(4):
            want = oc.eval(rlk, cts[b], Ts[:, b * 64:(b + 1) * 64], mode=mode, mask_seed=11 + b,
                           V=V[:, b * 64:(b + 1) * 64], group=og)
            assert np.array_equal(got[b], want), (mode, b)
        slots, budget = gc.decrypt(got)
        assert budget > 0 and slots.shape == (256,)
        if mode == 0:
            assert np.array_equal(slots, hashed) and int(slots.sum()) >= 9
        if mode == 1:
            assert int(slots.astype(np.int64).sum()) % T == int(hashed.sum())


def test_blocks_one_prime_response_batch_and_layers():
    oc, gc, s, rlk, sets, sid, Ts, V, cts, where, mu = _case(response_primes=1)
    cts2, _ = gc.query(sets.client[::-1].copy(), 9)
    outs = gc.eval_batch([sid, sid, sid], [cts, cts2, cts], [0, 1, 0], [0, 3, 0])
    for i, (c_, m_, s_) in enumerate(((cts, 0, 0), (cts2, 1, 3), (cts, 0, 0))):
        single = gc.eval(sid, c_, mode=m_, mask_seed=s_)
        assert single.shape == (4, 2, 1, 64) and np.array_equal(outs[i], single), i
        for b in range(4):
            want = oc.mod_switch(oc.eval(rlk, c_[b], Ts[:, b * 64:(b + 1) * 64], mode=m_, mask_seed=s_ + b), 1)
            assert np.array_equal(single[b], want), (i, b)
    gh, ge = gc.eval_layers(sid, cts, 1, 2)
    assert gh.shape == (4, 2, 2, 4, 64)
    for b in (0, 2):
        _, dh, de = oc.eval(rlk, cts[b], Ts[:, b * 64:(b + 1) * 64], layer0=1, nlayers=2, debug=True)
        assert np.array_equal(gh[b], dh) and np.array_equal(ge[b], de)


def test_bins_parameter_errors():
    import paper_2310_14565_gb300 as pepsi

    for bins in (32, 96, 64 * 3):
        with pytest.raises(pepsi.PepsiError):
            pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=4, bins=bins)
    gc = pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=4, bins=128)
    assert gc.blocks == 2 and gc.bins == 128
