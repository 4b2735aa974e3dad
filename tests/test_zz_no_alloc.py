"""pepsi_relin_noalloc: relinearisation for callers that cannot allocate
device memory (another allocator already holds it, or the caller's loop must
not pay for cudaMalloc / the synchronisation of cudaFree).  Its scratch is a
fixed 16 MiB device array inside the library, shared by all calls and left
holding the last call's contents.  Checked through the C ABI against
pepsi_relin, which allocates its scratch, and against the oracle's
relinearisation, on two calls in a row with different inputs: the second
call must not see stale words of the first.  At the paper size the largest
accepted batch fills the array exactly (8 ciphertexts at N = 8192, k = 4),
so the digit rows and the result rows placed after them reach its last word.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from gpu_helpers import T, pair, to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20


def _per_ct(k, N):
    return ((k + 2) + 2) * k * N * 8  # (k+2) digit rows and 2 result rows of k*N words


def _three_component_cts(oc, s, n, seed):
    rng = np.random.default_rng(seed)
    m = rng.integers(0, T, (2 * n, oc.N)).astype(np.uint32)
    cts = oc.encrypt(s, m, seed)
    return np.stack([oc.ct_mult(cts[i], cts[n + i]) for i in range(n)])


@pytest.mark.parametrize("N,bits,n", [(8192, [55, 55, 54, 54], 3), (8192, [55, 55, 54, 54], 8),
                                      (64, [36, 36, 37], 5)])
def test_relin_noalloc_matches_relin_and_oracle_on_two_calls(N, bits, n):
    torch_cuda()
    oc, gc, s, rlk = pair(N, bits, 1, 4, mu=1)
    assert n * _per_ct(oc.k, N) <= SCRATCH_BYTES
    for call, seed in enumerate((11, 12)):
        ct3h = _three_component_cts(oc, s, n, seed)
        ct3 = to_dev(ct3h)
        want = to_dev(np.zeros((n, 2, oc.k, N), np.uint64))
        gc.relin(ct3, n, want)
        got = to_dev(np.full((n, 2, oc.k, N), 7, np.uint64))
        gc.relin_noalloc(ct3, n, got)
        goth = to_host(got).reshape(n, 2, oc.k, N)
        assert np.array_equal(goth, to_host(want).reshape(n, 2, oc.k, N)), call
        for i in range(n):
            assert np.array_equal(goth[i], oc.relin(rlk, ct3h[i])), (call, i)
        slots, budget = oc.decrypt(s, goth[0])
        assert budget > 0


def test_relin_noalloc_rejects_oversized_requests():
    import paper_2310_14565_gb300 as pepsi

    torch_cuda()
    oc, gc, s, rlk = pair(8192, [55, 55, 54, 54], 1, 4, mu=1)
    n = SCRATCH_BYTES // _per_ct(4, 8192) + 1
    ct3 = to_dev(np.zeros((n, 3, 4, 8192), np.uint64))
    out = to_dev(np.zeros((n, 2, 4, 8192), np.uint64))
    with pytest.raises(pepsi.PepsiError) as e:
        gc.relin_noalloc(ct3, n, out)
    assert e.value.code == pepsi.E_PARAM and "bytes of scratch" in str(e.value)
    # a count whose byte size wraps 64 bits is rejected before any product:
    # the size check divides, so no buffer is touched (raw pointers, n huge)
    huge = (1 << 64) // _per_ct(4, 8192) + 1
    with pytest.raises(pepsi.PepsiError) as e:
        gc.relin_noalloc(ct3.data_ptr(), huge, out.data_ptr())
    assert e.value.code == pepsi.E_PARAM and "bytes of scratch" in str(e.value)
