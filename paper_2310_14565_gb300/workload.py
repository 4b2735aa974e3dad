"""Seeded synthetic item sets shaped like the paper's workloads.

The paper evaluates on random sets (Section 7): a client set X of m items
and a server set Y of n items, with a chosen number of items planted in
both.  This module holds no part of the method's arithmetic; it only draws
items, so the CUDA path and the CPU oracle can be fed identical inputs.

Recipe: numpy Generator(PCG64(seed)); server items uniform in [0, 2^bits),
distinct (repeated draws are redrawn); the planted items are a sample
without replacement of the server set written at random client positions;
the other client items are fresh uniform values not in the server set.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ItemSets:
    client: np.ndarray   # uint64 [m]
    server: np.ndarray   # uint64 [n]
    planted: np.ndarray  # uint64 [p], the items known to be in both


def _draw(rng, count, bits):
    if bits >= 64:
        return rng.integers(0, np.iinfo(np.uint64).max, size=count, dtype=np.uint64, endpoint=True)
    return rng.integers(0, 1 << bits, size=count, dtype=np.uint64)


def _unique_uniform(rng, count, bits, exclude=None):
    """count distinct uniform values in [0, 2^bits), none of them in exclude
    (a sorted uint64 array or None); collisions are redrawn."""
    out = _draw(rng, count, bits)
    while True:
        order = np.argsort(out, kind="stable")
        srt = out[order]
        bad = np.zeros(out.size, dtype=bool)
        if out.size > 1:
            bad[order[1:][srt[1:] == srt[:-1]]] = True  # later copies of a value are redrawn
        if exclude is not None and exclude.size and out.size:
            at = np.minimum(np.searchsorted(exclude, out), exclude.size - 1)
            bad |= exclude[at] == out
        nbad = int(bad.sum())
        if nbad == 0:
            return out
        out[bad] = _draw(rng, nbad, bits)


def make_sets(m: int, n: int, planted: int, bits: int = 64, seed_items: int = 1, seed_plant: int = 2) -> ItemSets:
    """Client set of m items, server set of n items, `planted` shared."""
    if planted > min(m, n):
        raise ValueError("cannot plant more items than either set holds")
    rng = np.random.Generator(np.random.PCG64(seed_items))
    server = _unique_uniform(rng, n, bits)
    rngp = np.random.Generator(np.random.PCG64(seed_plant))
    shared = server[np.sort(rngp.choice(n, size=planted, replace=False))] if planted else np.empty(0, np.uint64)
    fresh = _unique_uniform(rng, m - planted, bits, exclude=np.sort(server))
    client = np.concatenate([fresh, shared]).astype(np.uint64)
    pos = rngp.permutation(m)
    out = np.empty(m, dtype=np.uint64)
    out[pos] = client
    return ItemSets(client=out, server=server, planted=shared)


# Workloads of the configurations (sizes as in the paper's evaluation and
# its toy/large variants).
CONFIGS = {
    "toy": dict(N=4096, t=65537, prime_bits=[36, 36, 37], m=64, n=1024, planted=16, bits=32,
                lambda_bar=16, ell=363, h=2, mu=16),
    "paper": dict(N=8192, t=65537, prime_bits=[55, 55, 54, 54], m=1024, n=1 << 20, planted=102, bits=64,
                  lambda_bar=32, ell=600, h=4, mu=526),
    "large": dict(N=16384, t=65537, prime_bits=[55] * 6 + [54] * 2, m=4096, n=1 << 24, planted=41, bits=64,
                  lambda_bar=40, ell=128, h=8, mu=3487),
}
