"""Parity at the paper-shaped size, in the configuration bench.py times:
N = 8192, four 54/55-bit primes, t = 65537, h = 4, ell = 600, mu = 526,
1024 client items against 2^20 server items (102 planted), resident
server plaintexts, circuit chunks of 256 layers, one rounding of the
layers' last products per evaluation and a one-prime response.  The oracle
checks sampled outputs one by one (the server table, the request words,
sampled plaintexts, the h' and E words of sampled layers) and the whole
response of every mode word for word (about 80 s of oracle time each on
16 host cores); the result is also checked by properties that hold at any
size (decrypts to the brute-force intersection with positive budget, the
same as with per-layer rounding)."""
import numpy as np
import pytest

from gpu_helpers import brute_indicator, pair, torch_cuda

pytestmark = pytest.mark.gpu

PAPER = [55, 55, 54, 54]
ALL = 0xFFFFFFFF


@pytest.fixture(scope="module")
def paper_case():
    torch_cuda()
    from paper_2310_14565_gb300.workload import make_sets

    oc, gc, s, rlk = pair(8192, PAPER, 4, 32, mu=526, ell=600, rescale_group=ALL, server_values=1,
                          response_primes=1)
    sets = make_sets(1024, 1 << 20, 102, bits=64)
    gc.set_schedule(chunk=256)  # the chunk the autotuner picks at this size
    sid = gc.server_load(sets.server)
    rc, Ts, _ = oc.server_table(sets.server)
    assert rc == 0
    cts, where = gc.query(sets.client, 4)
    return oc, gc, s, rlk, sets, sid, Ts, cts, where


def _oracle_timed(oc, rlk, cts, Ts, mode=0, mask_seed=0, V=None):
    """The oracle's response in the timed configuration: one rounding of
    the last products of all 526 layers, switched to the first prime."""
    return oc.mod_switch(oc.eval(rlk, cts, Ts, mode=mode, mask_seed=mask_seed, group=526, V=V), 1)


@pytest.mark.parametrize("mode,mask_seed", [(0, 0), (1, 5)])
def test_paper_timed_configuration_words(paper_case, mode, mask_seed):
    """The whole response of the configuration bench.py times, word for word:
    256-layer chunks, so each k_tensor_sum launch sums 256 layers (64 per
    thread slice, through its periodic 128-bit reductions), lazy rescaling
    over all layers, a one-prime response; indicator and cardinality."""
    oc, gc, s, rlk, sets, sid, Ts, cts, where = paper_case
    assert gc.schedule()["chunk"] == 256
    got = gc.eval(sid, cts, mode=mode, mask_seed=mask_seed)
    want = _oracle_timed(oc, rlk, cts, Ts, mode, mask_seed)
    assert got.shape == want.shape == (2, 1, 8192)
    assert np.array_equal(got, want)


def test_paper_table_request_and_plaintexts(paper_case):
    oc, gc, s, rlk, sets, sid, Ts, cts, where = paper_case
    assert np.array_equal(gc.server_table(sid, 526), Ts)
    rc, ocs, owhere = oc.query(s, sets.client, 4)
    assert rc == 0 and np.array_equal(where, owhere)
    assert np.array_equal(cts, ocs)
    P = gc.server_plaintexts(sid, 263, 1)
    for j in (0, 299, 599):
        assert np.array_equal(P[0, j], oc.server_plaintext(Ts, 263, j))


def test_paper_sampled_layers(paper_case):
    oc, gc, s, rlk, sets, sid, Ts, cts, where = paper_case
    for layer0, nl in ((0, 2), (525, 1)):
        _, dh, de = oc.eval(rlk, cts, Ts, layer0=layer0, nlayers=nl, debug=True)
        gh, ge = gc.eval_layers(sid, cts, layer0, nl)
        assert np.array_equal(gh, dh), layer0
        assert np.array_equal(ge, de), layer0


def test_paper_result_decrypts_to_intersection(paper_case):
    oc, gc, s, rlk, sets, sid, Ts, cts, where = paper_case
    out = gc.eval(sid, cts)  # lazy rescaling, one-prime response (2 N words)
    assert out.shape == (2, 1, 8192)
    slots, budget = gc.decrypt(out)
    assert budget > 0
    assert np.array_equal(slots, brute_indicator(sets.client, sets.server, where, 8192))
    assert int(slots.sum()) == 102
    oslots, obudget = oc.decrypt(s, out)
    assert np.array_equal(oslots, slots) and abs(obudget - budget) < 1e-9
    # per-layer rounding on the same context and table decrypts the same
    gc.set_rescale_group(1)
    try:
        pslots, pbudget = gc.decrypt(gc.eval(sid, cts))
    finally:
        gc.set_rescale_group(ALL)
    assert pbudget > 0 and np.array_equal(pslots, slots)
    # the response switch of a full ciphertext, word for word
    assert np.array_equal(gc.mod_switch(cts[0], 1), oc.mod_switch(cts[0], 1))
    card = gc.eval(sid, cts, mode=1, mask_seed=5)
    cs, _ = gc.decrypt(card)
    assert int(cs.astype(np.int64).sum()) % 65537 == 102


def test_paper_labels_and_sum(paper_case):
    """Labelled PSI and PSI-Sum at the paper size: a second set, the same
    2^20 items with a value each; the labelled result decrypts to the value
    of every planted item at its bin and zero elsewhere, the masked sum to
    their total mod t."""
    oc, gc, s, rlk, sets, sid, Ts, cts, where = paper_case
    values = (np.arange(1 << 20, dtype=np.uint64) * 7919 % 65536 + 1).astype(np.uint32)
    vid = gc.server_load_values(sets.server, values)
    assert np.array_equal(gc.server_table(vid, 526), Ts)
    val_of = dict(zip(sets.server.tolist(), values.tolist()))
    want = np.zeros(8192, np.uint32)
    for u, x in enumerate(sets.client.tolist()):
        if x in val_of:
            want[where[u]] = val_of[x]
    labels = gc.eval(vid, cts, mode=2)
    slots, budget = gc.decrypt(labels)
    assert budget > 0 and np.array_equal(slots, want)
    total = gc.eval(vid, cts, mode=3, mask_seed=9)
    ss, budget = gc.decrypt(total)
    assert budget > 0 and int(ss.astype(np.int64).sum()) % 65537 == int(want.astype(np.int64).sum()) % 65537
    # both responses word for word against the oracle, in the timed configuration
    rc, Tv, V, _ = oc.server_table_values(sets.server, values)
    assert rc == 0 and np.array_equal(Tv, Ts)
    assert np.array_equal(gc.server_values(vid, 526), V)
    assert np.array_equal(labels, _oracle_timed(oc, rlk, cts, Ts, 2, 0, V))
    assert np.array_equal(total, _oracle_timed(oc, rlk, cts, Ts, 3, 9, V))


LARGE = [55] * 6 + [54] * 2


def test_large_config_streamed_plaintexts():
    """Large configuration: N = 16384, eight primes (438 bits), h = 8,
    ell = 128, mu = 3487, 4096 client items against 2^24 server items (1%
    planted).  The NTT-form plaintexts (468 GB) cannot be resident, so the
    evaluation regenerates them per layer chunk.  As bench.py runs it: one
    rounding of the layers' last products, a one-prime response.  The
    oracle checks the server table, the request words and one sampled
    layer's h' and E words; the result decrypts to the brute-force
    intersection."""
    torch_cuda()
    from paper_2310_14565_gb300.workload import make_sets

    oc, gc, s, rlk = pair(16384, LARGE, 8, 40, mu=3487, ell=128, rescale_group=ALL, response_primes=1)
    sets = make_sets(4096, 1 << 24, 41, bits=64)
    sid = gc.server_load(sets.server)
    rc, Ts, _ = oc.server_table(sets.server)
    assert rc == 0
    assert np.array_equal(gc.server_table(sid, 3487), Ts)
    cts, where = gc.query(sets.client, 4)
    rc, ocs, owhere = oc.query(s, sets.client, 4)
    assert rc == 0 and np.array_equal(where, owhere) and np.array_equal(cts, ocs)
    _, dh, de = oc.eval(rlk, cts, Ts, layer0=0, nlayers=1, debug=True)
    gh, ge = gc.eval_layers(sid, cts, 0, 1)
    assert np.array_equal(gh, dh) and np.array_equal(ge, de)
    out = gc.eval(sid, cts)
    slots, budget = gc.decrypt(out)
    assert budget > 0
    assert np.array_equal(slots, brute_indicator(sets.client, sets.server, where, 16384))
    assert int(slots.sum()) == 41


def test_paper_host_pieces_equal_device_request(paper_case):
    """A host request is multiplied in two pieces of code bits (the first 72 of
    600 bits here); a device request in one launch.  Same words."""
    torch = torch_cuda()
    oc, gc, s, rlk, sets, sid, Ts, cts, where = paper_case
    host = gc.eval(sid, cts)
    dev_in = torch.from_numpy(np.ascontiguousarray(cts).view(np.int64).copy()).cuda()
    dev_out = torch.zeros(host.size, dtype=torch.int64, device="cuda")
    gc.eval(sid, dev_in, out=dev_out)
    torch.cuda.synchronize()
    assert np.array_equal(dev_out.cpu().numpy().view(np.uint64).reshape(host.shape), host)
