"""The evaluation schedule (pepsi_set_schedule, pepsi_autotune) changes how
an evaluation is split into launches, never its words: every combination of
circuit chunk, threads per transform block, fused or stored
relinearisation, and batch tile and warp groups gives the oracle's words, for
h = 4 and h = 8 (the circuits with a relinearisation before the affine
step), with per-layer rounding and with one rounding for all layers."""
import itertools

import numpy as np
import pytest

from gpu_helpers import pair, torch_cuda

pytestmark = pytest.mark.gpu

PAPER = [55, 55, 54, 54]
LARGE = [55] * 6 + [54] * 2
ALL = 0xFFFFFFFF


@pytest.mark.parametrize("h,bits,lb,group", [(4, PAPER, 10, 1), (4, PAPER, 10, ALL), (8, LARGE, 12, ALL)])
def test_schedules_give_the_oracle_words(h, bits, lb, group):
    import oracle
    from paper_2310_14565_gb300.workload import make_sets

    torch_cuda()
    sets = make_sets(20, 90, 4, bits=32, seed_items=51, seed_plant=52)
    mu = max(9, oracle.simple_hash(0x5EED, lb, 6, sets.server, 1000)[2])
    oc, gc, s, rlk = pair(64, bits, h, lb, mu=mu, rescale_group=group)
    sid = gc.server_load(sets.server)
    rc, Ts, _ = oc.server_table(sets.server)
    assert rc == 0
    cts, _ = gc.query(sets.client, 4)
    cts2, _ = gc.query(sets.client[::-1].copy(), 5)
    want = oc.eval(rlk, cts, Ts, group=mu if group == ALL else 1)
    want2 = oc.eval(rlk, cts2, Ts, mode=1, mask_seed=3, group=mu if group == ALL else 1)
    for chunk, nt, fused in itertools.product((1, 4, 64), (0, 64, 256, 1024), (1, 0)):
        gc.set_schedule(chunk=chunk, ntt_threads=nt, relin_fused=fused)
        assert np.array_equal(gc.eval(sid, cts), want), (chunk, nt, fused)
    for bp, grp, br in itertools.product((32, 64), (1, 2), (1, 2, 3, 4)):
        gc.set_schedule(chunk=4, ntt_threads=0, relin_fused=1, batch_points=bp, batch_groups=grp, batch_requests=br)
        outs = gc.eval_batch([sid] * 4, [cts, cts2, cts, cts2], [0, 1, 0, 1], [0, 3, 0, 3])
        assert all(np.array_equal(outs[i], want if i % 2 == 0 else want2) for i in range(4)), (bp, grp, br)
    chunk = gc.autotune(sid, cts)
    sc = gc.schedule()
    assert sc["chunk"] == chunk and np.array_equal(gc.eval(sid, cts), want)


def test_schedule_rejects_out_of_range_fields():
    import paper_2310_14565_gb300 as pepsi

    torch_cuda()
    oc, gc, s, rlk = pair(64, PAPER, 4, 10, mu=4)
    for bad in (dict(chunk=0), dict(ntt_threads=48), dict(ntt_threads=2048), dict(relin_fused=2),
                dict(batch_points=16), dict(batch_groups=3), dict(batch_requests=5)):
        with pytest.raises(pepsi.PepsiError):
            gc.set_schedule(**bad)
    assert gc.schedule()["chunk"] >= 1
