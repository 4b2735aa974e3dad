"""pepsi_eval with device buffers can be captured into a CUDA graph once
its scratch exists (after one call): the captured launches replayed give
the same words as direct calls."""
import numpy as np
import pytest

from gpu_helpers import pair, to_host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("group", [0, 0xFFFFFFFF])
def test_eval_captured_in_a_cuda_graph(group):
    torch = torch_cuda()
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    sets = make_sets(20, 70, 4, bits=32, seed_items=81, seed_plant=82)
    mu = max(6, oracle.simple_hash(0x5EED, 10, 6, sets.server, 1000)[2])
    oc, gc, s, rlk = pair(64, [55, 55, 54, 54], 4, 10, mu=mu, rescale_group=group, response_primes=1)
    sid = gc.server_load(sets.server)
    cts_np, _ = gc.query(sets.client, 4)
    cts = torch.from_numpy(cts_np.view(np.int64)).cuda()
    out = torch.zeros((2, 1, 64), dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gc.eval(sid, cts, out=out, stream=stream)  # creates the scratch
    stream.synchronize()
    want = to_host(out).copy()
    graph = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        gc.eval(sid, cts, out=out, stream=torch.cuda.current_stream())
    for _ in range(3):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(to_host(out), want)
    _, Ts, _ = oc.server_table(sets.server)
    og = mu if group else 1
    assert np.array_equal(want, oc.mod_switch(oc.eval(rlk, cts_np, Ts, group=og), 1))


def test_autotune_picks_a_chunk_and_keeps_the_words():
    torch_cuda()
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    sets = make_sets(20, 90, 4, bits=32, seed_items=83, seed_plant=84)
    mu = max(20, oracle.simple_hash(0x5EED, 10, 6, sets.server, 1000)[2])
    oc, gc, s, rlk = pair(64, [55, 55, 54, 54], 4, 10, mu=mu, rescale_group=5)
    sid = gc.server_load(sets.server)
    cts, _ = gc.query(sets.client, 4)
    before = gc.eval(sid, cts)
    chunk = gc.autotune(sid, cts)
    # the balanced chunk sizes of the candidates for mu layers
    cands = set()
    for want in (32, 64, 128, 256, 512, 1024, 2048, 4096):
        parts = -(-mu // min(want, mu))
        cands.add(-(-mu // parts))
    assert chunk in cands and gc.schedule()["chunk"] == chunk
    assert np.array_equal(gc.eval(sid, cts), before)
    _, Ts, _ = oc.server_table(sets.server)
    assert np.array_equal(before, oc.eval(rlk, cts, Ts, group=5))
