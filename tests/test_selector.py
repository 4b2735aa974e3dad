"""Parameter selection of Section 6.1 (host-only C ABI calls; no GPU): the
request-size model against the values the paper prints."""
import json
import math
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _gold():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def pepsi():
    import paper_2310_14565_gb300 as p
    from paper_2310_14565_gb300 import build

    build.build()  # host-only calls: the library loads without a GPU
    return p


def test_comm_optimal_hamming_weight_matches_paper(pepsi):
    for row in _gold()["comm_optimal_h"]:
        assert pepsi.comm_optimal_h(row["lambda_bar"], row["bins"]) == row["h"], row["cite"]


def test_request_model_uses_table3_and_eq1(pepsi):
    g = _gold()
    for lo, hi, ln, lq in g["table3"]["rows"]:
        for h in (lo, hi):
            bits, ell, got_ln, got_lq = pepsi.request_bits(20, h, 4096)
            assert (got_ln, got_lq) == (ln, lq)
            # Eq. 1: ell is the smallest code length with C(ell, h) >= 2^20
            assert math.comb(ell, h) >= 1 << 20 and (ell == h or math.comb(ell - 1, h) < 1 << 20)
            assert bits == math.ceil(4096 / 2 ** ln) * ell * 2 ** ln * lq
    for row in g["code_length"]:
        assert pepsi.request_bits(row["lambda_bar"], row["h"], 8192)[1] == row["ell"], row["cite"]


def test_bins_above_n_take_more_blocks(pepsi):
    # ceil(b / N) blocks of N slots: h = 2 has N = 2^13
    b1 = pepsi.request_bits(32, 2, 8192)[0]
    assert pepsi.request_bits(32, 2, 8193)[0] == 2 * b1
    assert pepsi.request_bits(32, 2, 16384)[0] == 2 * b1


def test_tie_goes_to_the_smaller_weight(pepsi):
    # lambda_bar = 48: h = 23 and h = 24 give the same ell (52) and parameter set
    a, b = pepsi.request_bits(48, 23, 4096), pepsi.request_bits(48, 24, 4096)
    assert a[0] == b[0] and a[1] == b[1] == 52
    assert pepsi.comm_optimal_h(48, 4096) == 23
    assert pepsi.comm_optimal_h(48, 4096, h_max=22) < 23


def test_selector_errors(pepsi):
    for args in ((0, 2, 4096), (20, 0, 4096), (20, 65, 4096), (20, 2, 0), (63, 2, 4096)):
        with pytest.raises(pepsi.PepsiError):
            pepsi.request_bits(*args)
