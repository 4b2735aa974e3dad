"""Storage of the resident server plaintexts: 64-bit words (the default) or
7-byte words in three planes (every prime below 2^56).  The multiply-accumulate reads
either; both give the oracle's words, through single, piecewise-uploaded and
batched evaluations."""
import os

import numpy as np
import pytest

from gpu_helpers import T, to_dev, to_host, torch_cuda
from test_gpu_parity import PAPER, _psi_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bits,h,lb", [(PAPER, 4, 10), ([56, 56, 56], 4, 12), ([36, 36, 37], 2, 8)])
def test_seven_and_eight_byte_tables_give_the_oracle_words(bits, h, lb):
    torch_cuda()
    import paper_2310_14565_gb300 as pepsi

    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, bits, h, lb, mu=5, m=20, n=70, planted=4, chunk=3,
                                                          plaintext_bytes=7)
    assert gc.plaintext_bytes == 7
    mu = Ts.shape[0]
    os.environ["PEPSI_CHUNK"] = "3"
    try:
        g8 = pepsi.Context(N=64, t=T, prime_bits=bits, h=h, lambda_bar=lb, mu=mu, hash_key=0x5EED, key_seed=3)
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    assert g8.plaintext_bytes == 8
    sid8 = g8.server_load(sets.server)
    # the planes put back together are the oracle's NTT-form plaintexts
    P7, P8 = gc.server_plaintexts(sid, 0, mu), g8.server_plaintexts(sid8, 0, mu)
    assert np.array_equal(P7, P8)
    for l, j in ((0, 0), (mu - 1, gc.ell - 1), (mu // 2, 5)):
        assert np.array_equal(P7[l, j], oc.server_plaintext(Ts, l, j))
    want = oc.eval(rlk, cts, Ts)
    assert np.array_equal(gc.eval(sid, cts), want)  # host request: uploaded in pieces
    assert np.array_equal(g8.eval(sid8, cts), want)
    for g, i in ((gc, sid), (g8, sid8)):
        outs = g.eval_batch([i, i, i], [cts, cts, cts], [0, 1, 0], [0, 3, 0])
        assert np.array_equal(outs[0], want) and np.array_equal(outs[2], want)
        assert np.array_equal(outs[1], oc.eval(rlk, cts, Ts, mode=1, mask_seed=3))


def test_device_request_and_partial_residency_with_seven_bytes():
    """Device-resident request (one launch over all bits) and a table of
    which only a prefix is resident in the 7-byte format."""
    torch = torch_cuda()
    import paper_2310_14565_gb300 as pepsi

    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, PAPER, 4, 10, mu=7, m=20, n=70, planted=4, chunk=3,
                                                          plaintext_bytes=7)
    mu = Ts.shape[0]
    want = oc.eval(rlk, cts, Ts)
    out = torch.zeros(2 * gc.k * 64, dtype=torch.int64, device="cuda")
    gc.eval(sid, to_dev(cts), out=out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out).reshape(want.shape), want)
    per_layer7 = gc.ell * gc.k * 64 * 7
    os.environ["PEPSI_CHUNK"] = "3"
    try:
        g2 = pepsi.Context(N=64, t=T, prime_bits=PAPER, h=4, lambda_bar=10, mu=mu, hash_key=0x5EED, key_seed=3,
                           resident_bytes=per_layer7 * 3, plaintext_bytes=7)  # 3 of mu layers resident
    finally:
        os.environ.pop("PEPSI_CHUNK", None)
    sid2 = g2.server_load(sets.server)
    assert np.array_equal(g2.eval(sid2, cts), want)
    P = g2.server_plaintexts(sid2, 2, 1)  # last resident layer, from the planes
    assert np.array_equal(P[0, 7], oc.server_plaintext(Ts, 2, 7))
    P = g2.server_plaintexts(sid2, 3, 1)  # first regenerated layer
    assert np.array_equal(P[0, 7], oc.server_plaintext(Ts, 3, 7))


def test_wide_primes_keep_eight_bytes_and_bad_formats_are_refused():
    torch_cuda()
    import paper_2310_14565_gb300 as pepsi

    oc, gc, s, rlk, sets, Ts, cts, where, sid = _psi_case(64, [60, 60], 2, 8, mu=4, m=16, n=50, planted=3, chunk=2)
    assert gc.plaintext_bytes == 8
    assert np.array_equal(gc.eval(sid, cts), oc.eval(rlk, cts, Ts))
    for bits, pb in (([60, 60], 7), (PAPER, 5), (PAPER, 9)):
        with pytest.raises(pepsi.PepsiError) as e:
            pepsi.Context(N=64, t=T, prime_bits=bits, h=2, lambda_bar=8, mu=4, plaintext_bytes=pb)
        assert e.value.code == pepsi.E_PARAM
