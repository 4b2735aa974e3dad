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


def pair(N, bits, h, lambda_bar, mu, ell=0, hash_key=HASH_KEY, key_seed=KEY_SEED, resident_bytes=0):
    import oracle

    import paper_2310_14565_gb300 as pepsi

    oc = oracle.Ctx(N=N, t=T, prime_bits=bits, h=h, ell=ell, lambda_bar=lambda_bar, mu=mu, hash_key=hash_key)
    gc = pepsi.Context(N=N, t=T, prime_bits=bits, h=h, ell=ell, lambda_bar=lambda_bar, mu=mu, hash_key=hash_key,
                       key_seed=key_seed, resident_bytes=resident_bytes)
    s, rlk = oc.keygen(key_seed)
    return oc, gc, s, rlk


def brute_indicator(client, server, where, N):
    srv = set(int(x) for x in server)
    want = np.zeros(N, np.uint32)
    for u, x in enumerate(client):
        if int(x) in srv:
            want[where[u]] = 1
    return want
