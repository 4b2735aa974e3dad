"""CUDA path vs the CPU oracle, word for word, through the C ABI.

Integer work: every comparison is bit-exact (the noise budget, a float
derived from exact integers, is compared to 1e-9 bits).  Sizes span several
NTT tiles, ragged layer chunks and the edge cases of the method (empty sets,
all-dummy tables, the smallest ring).
"""
import math
import os

import numpy as np
import pytest

from gpu_helpers import T, brute_indicator, hashed_indicator, pair, to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu

TOY = [36, 36, 37]
PAPER = [55, 55, 54, 54]
LARGE = [55] * 6 + [54] * 2


@pytest.fixture(autouse=True)
def _cuda():
    torch_cuda()


# -------------------------------------------------------------- setup / keys
@pytest.mark.parametrize("N,bits,h,lb", [(16, TOY, 2, 6), (64, PAPER, 4, 10), (4096, TOY, 2, 16),
                                         (8192, PAPER, 4, 32), (16384, LARGE, 8, 40)])
def test_params_and_keys(N, bits, h, lb):
    oc, gc, s, rlk = pair(N, bits, h, lb, mu=4)
    assert gc.q == oc.q and gc.psi == oc.psi and gc.psi_t == oc.psi_t and gc.ell == oc.ell
    gs, grlk = gc.export_keys()
    assert np.array_equal(gs, s)
    assert np.array_equal(grlk, rlk)


# ------------------------------------------------------------------- NTT
@pytest.mark.parametrize("N,bits", [(16, TOY), (64, PAPER), (4096, TOY), (8192, PAPER), (16384, LARGE)])
def test_ntt_matches_oracle(N, bits):
    import oracle

    oc, gc, _, _ = pair(N, bits, 1, 4, mu=1)
    rng = np.random.default_rng(N)
    count = 3
    x = np.stack([np.stack([rng.integers(0, q, N, dtype=np.uint64) for q in oc.q]) for _ in range(count)])
    d = to_dev(x)
    gc.ntt(d, count)
    got = to_host(d).reshape(count, oc.k, N)
    for c in range(count):
        for p in range(oc.k):
            want = oracle.ntt_fwd(x[c, p], N, oc.q[p], oc.psi[p])
            assert np.array_equal(got[c, p], want), (c, p)
    gc.ntt(d, count, inverse=True)
    assert np.array_equal(to_host(d).reshape(x.shape), x)


# --------------------------------------------------------- client request
@pytest.mark.parametrize("N,bits,h,lb,m", [(64, TOY, 2, 8, 20), (4096, TOY, 2, 16, 64), (64, PAPER, 4, 10, 0)])
def test_query_matches_oracle(N, bits, h, lb, m):
    from paper_2310_14565_gb300.workload import make_sets

    oc, gc, s, _ = pair(N, bits, h, lb, mu=4)
    sets = make_sets(m, 64, min(m, 4), bits=32)
    rc, want, where_o = oc.query(s, sets.client, 4)
    assert rc == 0
    got, where = gc.query(sets.client, 4)
    assert np.array_equal(where, where_o[: len(where)])
    assert np.array_equal(got, want)
    # device output buffer, same words
    d = to_dev(np.zeros_like(want))
    gc.query(sets.client, 4, out=d)
    assert np.array_equal(to_host(d).reshape(want.shape), want)


# ------------------------------------------------------------ server side
@pytest.mark.parametrize("N,bits,h,lb,n,mu", [(64, TOY, 2, 8, 100, 16), (4096, TOY, 2, 16, 1024, 16),
                                              (64, PAPER, 4, 10, 0, 3)])
def test_server_table_and_plaintexts(N, bits, h, lb, n, mu):
    from paper_2310_14565_gb300.workload import make_sets

    oc, gc, _, _ = pair(N, bits, h, lb, mu=mu)
    sets = make_sets(0, n, 0, bits=32)
    rc, Ts, _ = oc.server_table(sets.server)
    assert rc == 0
    sid = gc.server_load(sets.server)
    assert np.array_equal(gc.server_table(sid, mu), Ts)
    got = gc.server_plaintexts(sid, 0, mu)
    rng = np.random.default_rng(1)
    for layer in sorted(set([0, mu - 1] + list(rng.integers(0, mu, 3)))):
        for j in sorted(set([0, oc.ell - 1] + list(rng.integers(0, oc.ell, 4)))):
            assert np.array_equal(got[layer, j], oc.server_plaintext(Ts, layer, j)), (layer, j)


# ---------------------------------------------------- ciphertext products
@pytest.mark.parametrize("N,bits", [(16, TOY), (64, PAPER), (4096, TOY), (64, LARGE), (8192, PAPER)])
def test_ct_mult_and_relin_match_oracle(N, bits):
    oc, gc, s, rlk = pair(N, bits, 1, 4, mu=1)
    rng = np.random.default_rng(7)
    n = 2
    m = rng.integers(0, T, (2 * n, N)).astype(np.uint32)
    cts = oc.encrypt(s, m, 9)
    a, b = cts[:n], cts[n:]
    da, db = to_dev(a), to_dev(b)
    out3 = to_dev(np.zeros((n, 3, oc.k, N), np.uint64))
    gc.ct_mult(da, db, n, out3)
    got3 = to_host(out3).reshape(n, 3, oc.k, N)
    out2 = to_dev(np.zeros((n, 2, oc.k, N), np.uint64))
    gc.ct_mult(da, db, n, out2, relin=True)
    got2 = to_host(out2).reshape(n, 2, oc.k, N)
    for i in range(n):
        want3 = oc.ct_mult(a[i], b[i])
        assert np.array_equal(got3[i], want3)
        assert np.array_equal(got2[i], oc.relin(rlk, want3))
    # squaring (a == b) takes the same path
    gc.ct_mult(da, da, n, out3)
    assert np.array_equal(to_host(out3).reshape(n, 3, oc.k, N)[0], oc.ct_mult(a[0], a[0]))


# -------------------------------------------------------------- evaluation
def _psi_case(N, bits, h, lb, mu, m, n, planted, chunk=None, seed=5, **ctx_kw):
    """A PSI instance; mu is raised to the actual maximum bin load."""
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    sets = make_sets(m, n, planted, bits=32, seed_items=seed, seed_plant=seed + 1)
    _, _, load = oracle.simple_hash(0x5EED, lb, int(math.log2(N)), sets.server, 10 * n + 1)
    mu = max(mu, load)
    if chunk:
        os.environ["PEPSI_CHUNK"] = str(chunk)
    try:
        oc, gc, s, rlk = pair(N, bits, h, lb, mu=mu, **ctx_kw)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    rc, Ts, _ = oc.server_table(sets.server)
    assert rc == 0
    rc, cts, where = oc.query(s, sets.client, 4)
    assert rc == 0
    sid = gc.server_load(sets.server)
    gcts, gwhere = gc.query(sets.client, 4)
    assert np.array_equal(gcts, cts)
    return oc, gc, s, rlk, sets, Ts, cts, where, sid


@pytest.mark.parametrize("h,bits,lb", [(1, TOY, 6), (2, TOY, 8), (4, PAPER, 10), (8, LARGE, 12)])
def test_eval_layers_match_oracle(h, bits, lb):
    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, bits, h, lb, mu=5, m=20, n=80, planted=5, chunk=2)
    mu = Ts.shape[0]
    want_out, dh, de = oc.eval(rlk, cts, Ts, debug=True)
    gh, ge = gc.eval_layers(sid, cts, 0, mu)
    assert np.array_equal(gh, dh)
    assert np.array_equal(ge, de)
    gh2, ge2 = gc.eval_layers(sid, cts, mu - 2, 2)  # a ragged sub-range
    assert np.array_equal(gh2, dh[mu - 2:]) and np.array_equal(ge2, de[mu - 2:])


@pytest.mark.parametrize("h,bits,lb,N", [(2, TOY, 8, 64), (4, PAPER, 10, 64), (8, LARGE, 12, 64), (2, TOY, 6, 16)])
def test_eval_matches_oracle_both_modes(h, bits, lb, N):
    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(N, bits, h, lb, mu=6, m=min(20, N // 2), n=70,
                                                          planted=4, chunk=4)
    hashed = hashed_indicator(sets.client, sets.server, where, N, lb)
    for mode in (0, 1):
        want = oc.eval(rlk, cts, Ts, mode=mode, mask_seed=5)
        got = gc.eval(sid, cts, mode=mode, mask_seed=5)
        assert np.array_equal(got, want), mode
        gslots, gb = gc.decrypt(got)
        oslots, ob = oc.decrypt(s, want)
        assert np.array_equal(gslots, oslots)
        assert abs(gb - ob) < 1e-9 and gb > 0
        if mode == 0:
            # exact in the hashed domain; contains every true member
            assert np.array_equal(gslots, hashed)
            true = brute_indicator(sets.client, sets.server, where, N)
            assert np.all(gslots >= true)
        else:
            assert int(gslots.astype(np.int64).sum()) % T == int(hashed.sum())


def test_eval_device_buffers_and_stream():
    torch = torch_cuda()
    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, PAPER, 4, 10, mu=4, m=16, n=60, planted=3)
    want = oc.eval(rlk, cts, Ts)
    dct = to_dev(cts)
    dout = to_dev(np.zeros((2, oc.k, 64), np.uint64))
    st = torch.cuda.Stream()
    gc.eval(sid, dct, out=dout, stream=st)
    st.synchronize()
    assert np.array_equal(to_host(dout).reshape(want.shape), want)
    slots, b = gc.decrypt(dout)
    assert np.array_equal(slots, oc.decrypt(s, want)[0])


def test_toy_config_full_parity():
    """Toy configuration: N=4096, 3 primes (36,36,37), h=2, ell=363, mu=16,
    64 client / 1024 server 32-bit items, 16 planted."""
    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(4096, TOY, 2, 16, mu=16, m=64, n=1024, planted=16)
    want = oc.eval(rlk, cts, Ts)
    got = gc.eval(sid, cts)
    assert np.array_equal(got, want)
    slots, b = gc.decrypt(got)
    assert b > 0
    assert np.array_equal(slots, brute_indicator(sets.client, sets.server, where, 4096))
    assert int(slots.sum()) == 16


# ------------------------------------------------------------- edge cases
def test_empty_sets_and_all_dummy_table():
    oc, gc, s, rlk = pair(64, TOY, 2, 8, mu=3)
    sid = gc.server_load(np.zeros(0, np.uint64))
    rc, Ts, _ = oc.server_table(np.zeros(0, np.uint64))
    assert (Ts == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    cts, where = gc.query(np.zeros(0, np.uint64), 4)
    rc, ocs, _ = oc.query(s, np.zeros(0, np.uint64), 4)
    assert np.array_equal(cts, ocs)
    got = gc.eval(sid, cts)
    assert np.array_equal(got, oc.eval(rlk, cts, Ts))
    slots, b = gc.decrypt(got)
    assert not slots.any() and b > 0


def test_protocol_failures_are_error_codes():
    import paper_2310_14565_gb300 as pepsi

    oc, gc, s, rlk = pair(16, TOY, 2, 6, mu=1)
    with pytest.raises(pepsi.PepsiError) as e:
        gc.server_load(np.arange(200, dtype=np.uint64))  # mu = 1 cannot hold 600 insertions into 16 bins
    assert e.value.code == pepsi.E_BIN_OVERFLOW
    with pytest.raises(pepsi.PepsiError) as e:
        gc.query(np.arange(17, dtype=np.uint64), 1)  # 17 items, 16 bins, no stash
    assert e.value.code == pepsi.E_CUCKOO_FAIL
    with pytest.raises(pepsi.PepsiError) as e:
        gc.eval(7, np.zeros((gc.ell, 2, gc.k, 16), np.uint64))
    assert e.value.code == pepsi.E_PARAM
    with pytest.raises(pepsi.PepsiError) as e:
        pepsi.Context(N=48, prime_bits=TOY)
    assert e.value.code == pepsi.E_PARAM
    with pytest.raises(pepsi.PepsiError) as e:
        pepsi.Context(N=64, prime_bits=TOY, h=3)
    assert e.value.code == pepsi.E_PARAM


def test_streamed_plaintexts_match_resident():
    """Server plaintexts regenerated per layer chunk (table not resident)
    give the same words as the resident table."""
    import paper_2310_14565_gb300 as pepsi

    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, PAPER, 4, 10, mu=6, m=20, n=70, planted=4, chunk=3)
    mu = Ts.shape[0]
    os.environ["PEPSI_CHUNK"] = "3"
    try:
        g2 = pepsi.Context(N=64, t=T, prime_bits=PAPER, h=4, lambda_bar=10, mu=mu, hash_key=0x5EED, key_seed=3,
                           resident_bytes=(1 << 64) - 1)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    sid2 = g2.server_load(sets.server)
    want = oc.eval(rlk, cts, Ts)
    assert np.array_equal(g2.eval(sid2, cts), want)
    assert np.array_equal(gc.eval(sid, cts), want)
    P = g2.server_plaintexts(sid2, 0, mu)
    assert np.array_equal(P[mu - 1, 3], oc.server_plaintext(Ts, mu - 1, 3))


@pytest.mark.parametrize("batch_points,batch_requests", [(32, 4), (64, 4), (32, 2)])
@pytest.mark.parametrize("resident", [True, False])
def test_eval_batch_matches_single_calls_and_oracle(resident, batch_points, batch_requests):
    """pepsi_eval_batch: two server sets, nine requests (with up to four
    requests per shared multiply-accumulate: groups of four and three on one
    set and of two on the other, so the shared multiply-accumulate runs for
    4, 3 and 2 requests; with up to two: pairs and a single), mixed modes and
    seeds, both tile widths of the shared multiply-accumulate; every output
    equals the single-request call and the oracle."""
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    N, bits, h, lb = 64, PAPER, 4, 10
    setsA = make_sets(20, 60, 4, bits=32, seed_items=11, seed_plant=12)
    setsB = make_sets(20, 50, 3, bits=32, seed_items=13, seed_plant=14)
    loads = [oracle.simple_hash(0x5EED, lb, 6, x.server, 1000)[2] for x in (setsA, setsB)]
    mu = max(loads)
    os.environ["PEPSI_CHUNK"] = "3"
    try:
        oc, gc, s, rlk = pair(N, bits, h, lb, mu=mu, resident_bytes=0 if resident else (1 << 64) - 1)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    gc.set_schedule(batch_points=batch_points, batch_requests=batch_requests)
    sA, sB = gc.server_load(setsA.server), gc.server_load(setsB.server)
    _, TA, _ = oc.server_table(setsA.server)
    _, TB, _ = oc.server_table(setsB.server)
    nreq = 9
    clients = [make_sets(16, 60, 3, bits=32, seed_items=20 + i, seed_plant=40 + i).client for i in range(nreq)]
    for i in (0, 3, 7):  # plant a few of A's items into three requests
        clients[i][:3] = setsA.server[:3]
    cts = [gc.query(cl, 100 + i)[0] for i, cl in enumerate(clients)]
    set_ids = [sA, sA, sB, sA, sA, sA, sB, sA, sA]
    modes = [0, 1, 0, 0, 1, 0, 1, 1, 0]
    seeds = [5, 6, 7, 8, 9, 10, 11, 12, 13]
    outs = gc.eval_batch(set_ids, cts, modes, seeds)
    for i in range(nreq):
        single = gc.eval(set_ids[i], cts[i], mode=modes[i], mask_seed=seeds[i])
        assert np.array_equal(outs[i], single), i
    for i in (0, 1, 2, 6, 7):
        T_ = TA if set_ids[i] == sA else TB
        assert np.array_equal(outs[i], oc.eval(rlk, cts[i], T_, mode=modes[i], mask_seed=seeds[i])), i
    slots, b = gc.decrypt(outs[0])
    assert b > 0 and int(slots.sum()) >= 3


def test_partially_resident_table():
    """A budget holding only some layers: the resident prefix and the
    regenerated rest give the words of the fully resident table."""
    import paper_2310_14565_gb300 as pepsi

    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, PAPER, 4, 10, mu=7, m=20, n=70, planted=4, chunk=3)
    mu = Ts.shape[0]
    per_layer = gc.ell * gc.k * 64 * 8
    os.environ["PEPSI_CHUNK"] = "3"
    try:
        g2 = pepsi.Context(N=64, t=T, prime_bits=PAPER, h=4, lambda_bar=10, mu=mu, hash_key=0x5EED, key_seed=3,
                           resident_bytes=per_layer * 4)  # 4 of mu layers resident
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    sid2 = g2.server_load(sets.server)
    want = oc.eval(rlk, cts, Ts)
    assert np.array_equal(g2.eval(sid2, cts), want)
    _, ge = g2.eval_layers(sid2, cts, 2, 4)  # straddles the resident boundary
    _, _, de = oc.eval(rlk, cts, Ts, debug=True)
    assert np.array_equal(ge, de[2:6])
    outs = g2.eval_batch([sid2, sid2], [cts, cts])
    assert np.array_equal(outs[0], want) and np.array_equal(outs[1], want)
    P = g2.server_plaintexts(sid2, 3, 2)
    assert np.array_equal(P[1, 0], oc.server_plaintext(Ts, 4, 0))


@pytest.mark.parametrize("h,bits,N", [(1, [36, 36], 64), (2, [48, 48, 48], 64), (4, [56, 56, 56], 64),
                                      (8, [51, 51, 51, 51], 64)])
def test_table3_prime_sets_match_oracle(h, bits, N):
    """The prime splits of Table 3's coefficient moduli (72, 144, 168, 204
    bits) used by the Hamming-weight sweep: words equal to the oracle."""
    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(N, bits, h, 12, mu=3, m=min(20, N // 2), n=40,
                                                          planted=3, chunk=2)
    want = oc.eval(rlk, cts, Ts)
    got = gc.eval(sid, cts)
    assert np.array_equal(got, want)
    slots, b = gc.decrypt(got)
    assert b > 0
    assert np.array_equal(slots, hashed_indicator(sets.client, sets.server, where, N, 12))


def test_host_request_uneven_pieces_match_oracle():
    """With more than 128 resident layers the first upload piece of a host
    request is shorter than half the code bits; the result is the oracle's."""
    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, PAPER, 4, 10, mu=160, m=20, n=70, planted=4, chunk=64)
    assert Ts.shape[0] >= 160 and gc.ell >= 8
    assert np.array_equal(gc.eval(sid, cts), oc.eval(rlk, cts, Ts))
