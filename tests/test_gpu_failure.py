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
