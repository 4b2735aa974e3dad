"""Modulus switching of the response (pepsi_mod_switch,
pepsi_params.response_primes) and decryption over the first r primes,
against the oracle word for word (the budget to 1e-9 bits)."""
import math
import os

import numpy as np
import pytest

from gpu_helpers import T, hashed_indicator, pair, to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu

TOY = [36, 36, 37]
PAPER = [55, 55, 54, 54]
LARGE = [55] * 6 + [54] * 2
ALL = 0xFFFFFFFF


@pytest.fixture(autouse=True)
def _cuda():
    torch_cuda()


@pytest.mark.parametrize("N,bits", [(64, TOY), (64, PAPER), (8192, PAPER), (16384, LARGE)])
def test_mod_switch_and_decrypt_match_oracle(N, bits):
    oc, gc, s, rlk = pair(N, bits, 1, 8, mu=2)
    rng = np.random.default_rng(N + len(bits))
    slots = rng.integers(0, T, size=(3, N)).astype(np.uint32)
    cts = oc.encrypt(s, np.stack([oc.encode(x) for x in slots]), 5)
    for r in sorted({1, 2, len(bits) - 1, len(bits)}):
        got = gc.mod_switch(cts, r)
        dev = to_host(gc.mod_switch(to_dev(cts), r, out=to_dev(np.zeros((3, 2, r, N), np.uint64))))
        for i in range(3):
            want = oc.mod_switch(cts[i], r)
            assert np.array_equal(got[i], want), (r, i)
            assert np.array_equal(dev[i], want), (r, i)
            gs, gb = gc.decrypt(got[i])
            os_, ob = oc.decrypt(s, want)
            assert np.array_equal(gs, os_) and np.array_equal(gs, slots[i])
            assert abs(gb - ob) < 1e-9 and gb > 0


@pytest.mark.parametrize("r", [1, 2])
@pytest.mark.parametrize("group", [0, ALL])
def test_eval_response_primes_matches_oracle(r, group):
    import oracle
    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300.workload import make_sets

    N, bits, h, lb = 64, PAPER, 4, 10
    sets = make_sets(20, 70, 5, bits=32, seed_items=41, seed_plant=42)
    values = np.random.default_rng(3).integers(1, T, size=70).astype(np.uint32)
    mu = max(7, oracle.simple_hash(0x5EED, lb, 6, sets.server, 1000)[2])
    oc, _, s, rlk = pair(N, bits, h, lb, mu=mu)
    os.environ["PEPSI_CHUNK"] = "3"
    try:
        gc = pepsi.Context(N=N, prime_bits=bits, h=h, lambda_bar=lb, mu=mu, hash_key=0x5EED, key_seed=3,
                           rescale_group=group, server_values=1, response_primes=r)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    assert gc.response_primes == r
    sid = gc.server_load_values(sets.server, values)
    _, Ts, V, _ = oc.server_table_values(sets.server, values)
    cts, where = gc.query(sets.client, 4)
    og = mu if group == ALL else 1
    hashed = hashed_indicator(sets.client, sets.server, where, N, lb)
    outs = gc.eval_batch([sid] * 4, [cts] * 4, [0, 1, 2, 3], [0, 5, 0, 6])
    for mode, seed, ob in zip((0, 1, 2, 3), (0, 5, 0, 6), outs):
        want = oc.mod_switch(oc.eval(rlk, cts, Ts, mode=mode, mask_seed=seed, V=V, group=og), r)
        got = gc.eval(sid, cts, mode=mode, mask_seed=seed)
        assert got.shape == (2, r, N)
        assert np.array_equal(got, want), mode
        assert np.array_equal(ob, want), mode
        sl, b = gc.decrypt(got)
        assert b > 0
        if mode == 0:
            assert np.array_equal(sl, hashed)


def test_response_primes_errors():
    import paper_2310_14565_gb300 as pepsi

    with pytest.raises(pepsi.PepsiError):
        pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=4, response_primes=5)
    gc = pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=4)
    with pytest.raises(pepsi.PepsiError):
        gc.mod_switch(np.zeros((2, 4, 64), np.uint64), 0)
    with pytest.raises(pepsi.PepsiError):
        gc.mod_switch(np.zeros((2, 4, 64), np.uint64), 5)
