"""The restatement of the device's parallel cuckoo rounds that the GPU test
compares with, pinned on its own: a valid, deterministic placement."""
import numpy as np
import pytest


@pytest.mark.parametrize("gamma,bins,load", [(1, 64, 0.85), (2, 64, 0.9), (3, 32, 0.9), (1, 256, 0.7)])
def test_parallel_cuckoo_rounds_restatement_is_a_valid_placement(gamma, bins, load):
    """The test restatement of the device cuckoo rounds places every item in
    one of its three candidate bins, at most gamma per bin, deterministically;
    with more items than slots it gives up."""
    from cuckoo_rounds import rounds_reference

    rng = np.random.default_rng(7 + gamma + bins)
    m = int(load * gamma * bins)
    cand = [list(rng.integers(0, bins, 3)) for _ in range(m)]
    where = rounds_reference(cand, gamma, bins)
    assert where is not None and where == rounds_reference(cand, gamma, bins)
    assert len(set(where)) == m
    per_bin = {}
    for u, w in enumerate(where):
        assert w // gamma in cand[u]
        per_bin[w // gamma] = per_bin.get(w // gamma, 0) + 1
    assert max(per_bin.values()) <= gamma
    over = [list(rng.integers(0, 4, 3)) for _ in range(4 * gamma + 1)]
    assert rounds_reference(over, gamma, 4, max_rounds=200) is None
