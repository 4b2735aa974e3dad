"""Shared helpers of the GPU parity tests: paired oracle / CUDA contexts and
device buffers.  The oracle and the CUDA path receive the same parameters and
seeds; their outputs are compared word for word."""
import numpy as np
import pytest

T = 65537
HASH_KEY = 0x5EED
KEY_SEED = 3


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available: the gpu tests need a GB300")
    return torch


def to_dev(arr):
    torch = torch_cuda()
    a = np.ascontiguousarray(arr, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def to_host(t):
    return t.cpu().numpy().view(np.uint64)


def pair(N, bits, h, lambda_bar, mu, ell=0, hash_key=HASH_KEY, key_seed=KEY_SEED, resident_bytes=0, rescale_group=0,
         **ctx_kw):
    import oracle

    import paper_2310_14565_gb300 as pepsi

    oc = oracle.Ctx(N=N, t=T, prime_bits=bits, h=h, ell=ell, lambda_bar=lambda_bar, mu=mu, hash_key=hash_key)
    gc = pepsi.Context(N=N, t=T, prime_bits=bits, h=h, ell=ell, lambda_bar=lambda_bar, mu=mu, hash_key=hash_key,
                       key_seed=key_seed, resident_bytes=resident_bytes, rescale_group=rescale_group, **ctx_kw)
    s, rlk = oc.keygen(key_seed)
    return oc, gc, s, rlk


def brute_indicator(client, server, where, N):
    """Slot indicator of the plain intersection X ∩ Y (client item u sits in
    slot where[u])."""
    srv = set(int(x) for x in server)
    want = np.zeros(N, np.uint32)
    for u, x in enumerate(client):
        if int(x) in srv:
            want[where[u]] = 1
    return want


def hashed_indicator(client, server, where, N, lambda_bar, hash_key=HASH_KEY):
    """Slot indicator the method decides exactly (Section 4): the client item
    in bin beta with low part x_L matches when some server item y has y_L =
    x_L and beta among y's three bins.  It contains the plain intersection;
    it differs from it only by H0 collisions at rate about 2^-lambda_bar per
    comparison, which small test values of lambda_bar make visible.  Brute
    force over the server items, with the oracle's item hash."""
    import oracle

    logb = int(N).bit_length() - 1
    by_low = {}
    for y in server:
        yl, bins = oracle.hash_item(hash_key, lambda_bar, logb, int(y))
        by_low.setdefault(yl, set()).update(int(b) for b in bins)
    want = np.zeros(N, np.uint32)
    for u, x in enumerate(client):
        if where[u] < 0:
            continue
        xl, _ = oracle.hash_item(hash_key, lambda_bar, logb, int(x))
        if int(where[u]) in by_low.get(xl, ()):
            want[where[u]] = 1
    return want
