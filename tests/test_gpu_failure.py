"""Failure detection without a GPU fault: a bounded device wait that
nothing completes gives up (about one second), the kernel reports it
through the context's error word, the call returns PEPSI_E_TIMEOUT, and the
context keeps working."""
import time

import numpy as np
import pytest

from gpu_helpers import pair, torch_cuda

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_recovers():
    torch_cuda()
    import oracle
    import paper_2310_14565_gb300 as pepsi
    from paper_2310_14565_gb300.workload import make_sets

    oc, gc, s, rlk = pair(64, [55, 55, 54, 54], 4, 10, mu=6)
    assert gc.wait_probe(1) == pepsi.OK
    t0 = time.perf_counter()
    assert gc.wait_probe(0) == pepsi.E_TIMEOUT
    waited = time.perf_counter() - t0
    assert 0.5 < waited < 30.0
    assert gc.wait_probe(1) == pepsi.OK  # the error word was cleared
    sets = make_sets(16, 40, 3, bits=32, seed_items=7, seed_plant=8)
    mu = max(6, oracle.simple_hash(0x5EED, 10, 6, sets.server, 1000)[2])
    oc, gc, s, rlk = pair(64, [55, 55, 54, 54], 4, 10, mu=mu)
    assert gc.wait_probe(0) == pepsi.E_TIMEOUT
    sid = gc.server_load(sets.server)
    cts, _ = gc.query(sets.client, 4)
    _, Ts, _ = oc.server_table(sets.server)
    assert np.array_equal(gc.eval(sid, cts), oc.eval(rlk, cts, Ts))


def test_binding_rejects_malformed_sizes():
    """Buffers smaller than the documented layouts never reach the C ABI
    (whose raw pointers cannot be checked), so no kernel reads or writes
    past them."""
    torch = torch_cuda()
    import paper_2310_14565_gb300 as pepsi

    gc = pepsi.Context(N=64, prime_bits=[55, 55, 54, 54], h=4, lambda_bar=10, mu=4)
    sid = gc.server_load(np.arange(1, 20, dtype=np.uint64))
    good = np.zeros((gc.ell, 2, 4, 64), np.uint64)
    short = torch.zeros(gc.ell * 2 * 4 * 64 - 1, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        gc.eval(sid, short)
    with pytest.raises(ValueError):
        gc.eval(sid, good, out=np.zeros((2, 4, 63), np.uint64))
    with pytest.raises(ValueError):
        gc.eval(sid, good.astype(np.uint32))  # 4-byte words
    with pytest.raises(ValueError):
        gc.eval_batch([sid], [short])
    with pytest.raises(ValueError):
        gc.decrypt(np.zeros((2, 4, 32), np.uint64))
    with pytest.raises(ValueError):
        gc.ntt(torch.zeros(3 * 4 * 64 - 8, dtype=torch.int64, device="cuda"), 3)
    one = torch.zeros(2 * 4 * 64, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        gc.ct_mult(one, one[:-1], 1, torch.zeros(3 * 4 * 64, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        gc.ct_mult(one, one, 1, torch.zeros(3 * 4 * 64 - 1, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        gc.mod_switch(np.zeros((2, 4, 64), np.uint64), 1, out=np.zeros((2, 1, 60), np.uint64))
    out = gc.eval(sid, gc.query(np.arange(5, 9, dtype=np.uint64), 4)[0])  # well-formed calls still work
    assert gc.decrypt(out)[1] > 0
