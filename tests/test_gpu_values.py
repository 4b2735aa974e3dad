"""Labelled PSI (Algorithm 4) and PSI-Sum (Algorithm 5) through the C ABI
against the oracle, word for word: the value table, both modes with
per-layer rounding and with lazy rescaling (and its per-layer fallback when
the auxiliary base has no room for the value products), streamed
plaintexts, batches mixing all four modes, and the protocol errors."""
import math
import os

import numpy as np
import pytest

from gpu_helpers import T, pair, torch_cuda

pytestmark = pytest.mark.gpu

TOY = [36, 36, 37]
PAPER = [55, 55, 54, 54]
LARGE = [55] * 6 + [54] * 2
ALL = 0xFFFFFFFF


@pytest.fixture(autouse=True)
def _cuda():
    torch_cuda()


def _labels(oracle, client, where, Ts, V, lb, N):
    """Expected labelled result: per client slot, the value stored with the
    same x_L in that bin (hashed domain), else 0."""
    out = np.zeros(N, np.uint32)
    for u, x in enumerate(client):
        if where[u] < 0:
            continue
        xl, _ = oracle.hash_item(0x5EED, lb, int(math.log2(N)), int(x))
        hit = np.nonzero(Ts[:, where[u]] == xl)[0]
        if hit.size:
            out[where[u]] = V[hit[0], where[u]]
    return out


def _case(N, bits, h, lb, group=0, server_values=0, chunk=4, resident_bytes=0, seed=31):
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    sets = make_sets(20, 70, 5, bits=32, seed_items=seed, seed_plant=seed + 1)
    values = np.random.default_rng(seed).integers(1, T, size=70).astype(np.uint32)
    load = oracle.simple_hash(0x5EED, lb, int(math.log2(N)), sets.server, 1000)[2]
    mu = max(7, load)
    os.environ["PEPSI_CHUNK"] = str(chunk)
    try:
        oc, gc, s, rlk = pair(N, bits, h, lb, mu=mu, resident_bytes=resident_bytes, rescale_group=group)
        if server_values:
            import paper_2310_14565_gb300 as pepsi

            gc = pepsi.Context(N=N, t=T, prime_bits=bits, h=h, lambda_bar=lb, mu=mu, hash_key=0x5EED, key_seed=3,
                               resident_bytes=resident_bytes, rescale_group=group, server_values=1)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    rc, Ts, V, _ = oc.server_table_values(sets.server, values)
    assert rc == 0
    sid = gc.server_load_values(sets.server, values)
    cts, where = gc.query(sets.client, 4)
    labels = _labels(oracle, sets.client, where, Ts, V, lb, N)
    return oc, gc, s, rlk, sets, Ts, V, cts, where, sid, mu, labels


def test_value_table_matches_oracle():
    oc, gc, s, rlk, sets, Ts, V, cts, where, sid, mu, labels = _case(64, PAPER, 4, 10)
    assert np.array_equal(gc.server_table(sid, mu), Ts)
    assert np.array_equal(gc.server_values(sid, mu), V)
    assert int((labels != 0).sum()) >= 5


@pytest.mark.parametrize("rounding", ["layer", "lazy", "lazy-no-room"])
@pytest.mark.parametrize("h,bits,lb", [(1, TOY, 8), (2, TOY, 8), (4, PAPER, 10), (8, LARGE, 12)])
def test_labels_and_sum_match_oracle(h, bits, lb, rounding):
    group = 0 if rounding == "layer" else ALL
    oc, gc, s, rlk, sets, Ts, V, cts, where, sid, mu, labels = _case(64, bits, h, lb, group=group,
                                                                     server_values=rounding == "lazy")
    og = mu if (rounding == "lazy" and h > 1) else 1
    for mode in (2, 3):
        want = oc.eval(rlk, cts, Ts, mode=mode, mask_seed=7, V=V, group=og)
        got = gc.eval(sid, cts, mode=mode, mask_seed=7)
        assert np.array_equal(got, want), mode
        slots, b = gc.decrypt(got)
        assert b > 0
        if mode == 2:
            assert np.array_equal(slots, labels)
        else:
            assert int(slots.astype(np.int64).sum()) % T == int(labels.astype(np.int64).sum()) % T
    # the plain modes on a set with values are unchanged
    assert np.array_equal(gc.eval(sid, cts), oc.eval(rlk, cts, Ts, group=mu if rounding != "layer" else 1))


@pytest.mark.parametrize("group", [0, 3])
def test_values_streamed_plaintexts(group):
    oc, gc, s, rlk, sets, Ts, V, cts, where, sid, mu, labels = _case(64, PAPER, 4, 10, group=group,
                                                                     server_values=1, chunk=3,
                                                                     resident_bytes=(1 << 64) - 1)
    og = 3 if group == 3 else 1
    got = gc.eval(sid, cts, mode=2)
    assert np.array_equal(got, oc.eval(rlk, cts, Ts, mode=2, V=V, group=og))
    assert np.array_equal(gc.decrypt(got)[0], labels)


@pytest.mark.parametrize("group", [0, ALL])
def test_values_batch_mixed_modes(group):
    oc, gc, s, rlk, sets, Ts, V, cts, where, sid, mu, labels = _case(64, PAPER, 4, 10, group=group,
                                                                     server_values=1, chunk=3)
    cts2, _ = gc.query(sets.client[::-1].copy(), 9)
    reqs = [cts, cts2, cts, cts2]
    modes = [2, 3, 0, 1]
    seeds = [0, 6, 0, 8]
    outs = gc.eval_batch([sid] * 4, reqs, modes, seeds)
    og = mu if group == ALL else 1
    for i in range(4):
        assert np.array_equal(outs[i], gc.eval(sid, reqs[i], mode=modes[i], mask_seed=seeds[i])), i
        assert np.array_equal(outs[i], oc.eval(rlk, reqs[i], Ts, mode=modes[i], mask_seed=seeds[i], V=V,
                                               group=og)), i


def test_value_mode_errors():
    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300.workload import make_sets

    gc = pepsi.Context(N=64, prime_bits=PAPER, h=4, lambda_bar=10, mu=8, hash_key=0x5EED)
    sets = make_sets(10, 30, 2, bits=32, seed_items=3, seed_plant=4)
    plain = gc.server_load(sets.server)
    cts, _ = gc.query(sets.client, 4)
    for mode in (2, 3):
        with pytest.raises(pepsi.PepsiError) as ei:
            gc.eval(plain, cts, mode=mode)
        assert ei.value.code == pepsi.E_PARAM
    with pytest.raises(pepsi.PepsiError) as ei:
        gc.eval(plain, cts, mode=4)
    assert ei.value.code == pepsi.E_PARAM
    bad = np.full(30, T, np.uint32)  # a value must be below t
    with pytest.raises(pepsi.PepsiError) as ei:
        gc.server_load_values(sets.server, bad)
    assert ei.value.code == pepsi.E_PARAM
    with pytest.raises(pepsi.PepsiError):
        gc.server_values(plain, 8)
    empty = gc.server_load_values(np.zeros(0, np.uint64), np.zeros(0, np.uint32))
    out = gc.eval(empty, cts, mode=2)
    slots, b = gc.decrypt(out)
    assert b > 0 and not slots.any()
