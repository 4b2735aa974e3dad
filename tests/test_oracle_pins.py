"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value
printed in the paper, a library routine (sympy / scipy), a closed form, an
invariant, or brute force on tiny inputs.  None of these needs a GPU.
"""
import itertools
import json
import math
import os
import random

import numpy as np
import pytest
import sympy
from sympy.ntheory.modular import crt as sympy_crt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
T = 65537


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def brev(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


def negacyclic_schoolbook(a, b, N, mod=None):
    out = [0] * N
    for i in range(N):
        for j in range(N):
            p = a[i] * b[j]
            if i + j >= N:
                out[i + j - N] -= p
            else:
                out[i + j] += p
    return [x % mod for x in out] if mod else out


# ------------------------------------------------------------ primes, roots
def test_miller_rabin_matches_sympy(oracle_mod):
    rng = random.Random(1)
    cands = [rng.getrandbits(64) | 1 for _ in range(300)] + [2, 3, 4, 65537, 2**61 - 1, 2**64 - 59, 3215031751]
    for n in cands:
        assert oracle_mod.is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("bits,N", [(36, 4096), (37, 4096), (55, 8192), (54, 8192), (55, 16384), (20, 16)])
def test_prime_search_is_largest(oracle_mod, bits, N):
    q = oracle_mod.find_prime(bits, N)
    assert q % (2 * N) == 1 and sympy.isprime(q) and q < 2**bits
    # no prime = 1 mod 2N lies between q and 2^bits
    for c in range(q + 2 * N, 2**bits, 2 * N):
        assert not sympy.isprime(c)
    q2 = oracle_mod.find_prime(bits, N, [q])
    assert q2 < q and sympy.isprime(q2)
    for c in range(q2 + 2 * N, q, 2 * N):
        assert not sympy.isprime(c)


def test_min_root_brute_force(oracle_mod):
    for N in (4, 8, 16):
        q = oracle_mod.find_prime(14, N)
        roots = [w for w in range(1, q) if pow(w, N, q) == q - 1]
        assert oracle_mod.min_root(q, N) == min(roots)
    # t = 65537: the minimal primitive 2N-th root
    for N in (16, 64):
        r = oracle_mod.min_root(T, N)
        assert pow(r, N, T) == T - 1
        assert all(pow(w, N, T) != T - 1 for w in range(1, r))


# ------------------------------------------------------------------ NTT
@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
def test_ntt_matches_evaluation_definition(oracle_mod, N):
    q = oracle_mod.find_prime(40, N)
    psi = oracle_mod.min_root(q, N)
    rng = random.Random(N)
    a = [rng.randrange(q) for _ in range(N)]
    lg = int(math.log2(N))
    want = [sum(a[n] * pow(psi, (2 * brev(i, lg) + 1) * n, q) for n in range(N)) % q for i in range(N)]
    assert [int(x) for x in oracle_mod.ntt_fwd(a, N, q, psi)] == want
    assert [int(x) for x in oracle_mod.ntt_direct(a, N, q, psi)] == want
    assert [int(x) for x in oracle_mod.ntt_inv(want, N, q, psi)] == a


@pytest.mark.parametrize("N,bits", [(8, 55), (32, 61), (64, 36)])
def test_ntt_product_is_negacyclic_convolution(oracle_mod, N, bits):
    q = oracle_mod.find_prime(bits, N)
    psi = oracle_mod.min_root(q, N)
    rng = random.Random(bits)
    a = [rng.randrange(q) for _ in range(N)]
    b = [rng.randrange(q) for _ in range(N)]
    A = oracle_mod.ntt_fwd(a, N, q, psi)
    B = oracle_mod.ntt_fwd(b, N, q, psi)
    prod = [int(x) * int(y) % q for x, y in zip(A, B)]
    got = [int(x) for x in oracle_mod.ntt_inv(prod, N, q, psi)]
    assert got == negacyclic_schoolbook(a, b, N, q)


def test_crt_matches_sympy(oracle_mod):
    rng = random.Random(5)
    for k in (1, 3, 8, 16):
        ps = []
        for _ in range(k):
            ps.append(oracle_mod.find_prime(61 if k > 8 else 55, 64, ps))
        x = rng.randrange(math.prod(ps))
        res = [x % p for p in ps]
        assert oracle_mod.crt(res, ps) == int(sympy_crt(ps, res)[0]) == x


# ------------------------------------------------------- batch encoding
def test_encoding_is_evaluation_at_odd_powers(oracle_mod):
    N = 32
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=[36], h=1, lambda_bar=4)
    rng = random.Random(2)
    m = [rng.randrange(T) for _ in range(N)]
    slots = c.decode(np.array(m, np.uint32))
    want = [sum(m[n] * pow(c.psi_t, (2 * s + 1) * n, T) for n in range(N)) % T for s in range(N)]
    assert [int(x) for x in slots] == want
    assert [int(x) for x in c.encode(slots)] == m


def test_encoding_is_a_ring_homomorphism(oracle_mod):
    N = 16
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=[36], h=1, lambda_bar=4)
    rng = random.Random(3)
    a = [rng.randrange(T) for _ in range(N)]
    b = [rng.randrange(T) for _ in range(N)]
    ab = negacyclic_schoolbook(a, b, N, T)
    da, db, dab = (c.decode(np.array(x, np.uint32)) for x in (a, b, ab))
    assert [int(x) for x in dab] == [int(x) * int(y) % T for x, y in zip(da, db)]
    # a constant polynomial puts the constant in every slot
    assert set(int(x) for x in c.decode(np.array([7] + [0] * (N - 1), np.uint32))) == {7}


# ------------------------------------------------------------ the code
def test_code_length_paper_value(oracle_mod):
    for row in golden("paper_values.json")["code_length"]:
        assert oracle_mod.code_length(row["lambda_bar"], row["h"]) == row["ell"]


@pytest.mark.parametrize("lb,h", [(16, 2), (32, 4), (40, 8), (19, 8), (10, 1), (32, 2)])
def test_code_length_is_minimal(oracle_mod, lb, h):
    ell = oracle_mod.code_length(lb, h)
    assert math.comb(ell, h) >= 2**lb > math.comb(ell - 1, h)


@pytest.mark.parametrize("ell,h", [(6, 2), (8, 3), (10, 4), (9, 1), (12, 8)])
def test_cw_encode_is_colex_unranking(oracle_mod, ell, h):
    combos = sorted(itertools.combinations(range(ell), h), key=lambda c: tuple(reversed(c)))
    assert len(combos) == math.comb(ell, h)
    for v, combo in enumerate(combos):
        pos = oracle_mod.cw_encode(v, ell, h)
        assert tuple(pos) == combo
        assert sum(math.comb(c, r + 1) for r, c in enumerate(pos)) == v
    with pytest.raises(ValueError):
        oracle_mod.cw_encode(len(combos), ell, h)


# ----------------------------------------------------------- randomness
def test_splitmix64_published_outputs(oracle_mod):
    g = golden("splitmix64.json")["state0_outputs"]
    gamma = 0x9E3779B97F4A7C15
    for i, want in enumerate(g):
        assert oracle_mod.mix64((i + 1) * gamma % 2**64) == int(want, 16)


def test_samplers_distribution(oracle_mod):
    st = oracle_mod.stream(1, 0, 0)
    tern = [oracle_mod.sample_mod(9, st, i, 3) for i in range(30000)]
    counts = np.bincount(tern, minlength=3) / len(tern)
    assert np.all(np.abs(counts - 1 / 3) < 0.02)
    cbd = np.array([oracle_mod.sample_cbd(9, st, i) for i in range(30000)])
    assert cbd.min() >= -21 and cbd.max() <= 21
    assert abs(cbd.mean()) < 0.1 and abs(cbd.var() - 10.5) < 0.5
    q = 2**55 - 2**20 + 1
    u = np.array([oracle_mod.sample_mod(9, st, i, q) for i in range(5000)], dtype=np.float64)
    assert u.max() < q and abs(u.mean() / q - 0.5) < 0.02


# ----------------------------------------------------------------- hashing
def test_cuckoo_invariants(oracle_mod):
    rng = np.random.default_rng(4)
    items = np.unique(rng.integers(0, 2**32, 900, dtype=np.uint64))[:800]
    rc, table, where = oracle_mod.cuckoo(77, 16, 10, items)
    assert rc == 0
    assert len(set(where.tolist())) == len(items)
    for u, x in enumerate(items):
        xl, bins = oracle_mod.hash_item(77, 16, 10, x)
        assert where[u] in bins and table[where[u]] == xl
    assert int((table != oracle_mod.DUMMY).sum()) == len(items)
    # more items than bins cannot be placed: failure, not a hang
    rc, _, _ = oracle_mod.cuckoo(77, 16, 4, np.arange(17, dtype=np.uint64))
    assert rc == oracle_mod.E_CUCKOO_FAIL


@pytest.mark.parametrize("gamma", [2, 3])
def test_bucketed_cuckoo_invariants(oracle_mod, gamma):
    """Client bins of gamma slots (the client's maximum bin load, Section 4):
    more items than bins are placed; every item sits in a slot of one of its
    three bins with its x_L; no slot holds two items; a bin's occupied slots
    are its first ones (new items take the first free slot, evictions
    replace in place); gamma = 1 gives the one-slot table."""
    rng = np.random.default_rng(14 + gamma)
    b, logb = 256, 8
    items = np.unique(rng.integers(0, 2**32, 2 * b, dtype=np.uint64))[: int(0.8 * gamma * b)]
    rc, table, where = oracle_mod.cuckoo(77, 16, logb, items, gamma)
    assert rc == 0 and len(items) > b and table.shape == (b * gamma,)
    assert len(set(where.tolist())) == len(items)
    for u, x in enumerate(items):
        xl, bins = oracle_mod.hash_item(77, 16, logb, x)
        assert where[u] // gamma in bins and table[where[u]] == xl
    occ = (table != oracle_mod.DUMMY).reshape(b, gamma)
    assert int(occ.sum()) == len(items)
    for row in occ:
        n = int(row.sum())
        assert row[:n].all() and not row[n:].any()
    # the gamma = 1 table is the one-slot cuckoo of the same items, where it fits
    few = items[: b // 2]
    r1, t1, w1 = oracle_mod.cuckoo(77, 16, logb, few)
    rg, tg, wg = oracle_mod.cuckoo(77, 16, logb, few, 1)
    assert r1 == rg == 0 and np.array_equal(t1, tg) and np.array_equal(w1, wg)
    # more items than the gamma * b slots cannot be placed: failure, not a hang
    rc, _, _ = oracle_mod.cuckoo(77, 16, 4, np.arange(16 * gamma + 1, dtype=np.uint64), gamma)
    assert rc == oracle_mod.E_CUCKOO_FAIL


def test_simple_hash_invariants(oracle_mod):
    rng = np.random.default_rng(5)
    items = np.unique(rng.integers(0, 2**32, 3000, dtype=np.uint64))
    rc, Ts, mx = oracle_mod.simple_hash(13, 12, 8, items, 64)
    assert rc == 0 and mx <= 64
    expect = [[] for _ in range(256)]
    for x in items:
        xl, bins = oracle_mod.hash_item(13, 12, 8, x)
        for i, b in enumerate(bins):
            if b in bins[:i] or xl in expect[b]:
                continue
            expect[b].append(xl)
    for b in range(256):
        col = [int(v) for v in Ts[:, b] if v != oracle_mod.DUMMY]
        assert col == expect[b]
        assert all(v == oracle_mod.DUMMY for v in Ts[len(col):, b])
    rc, _, mx2 = oracle_mod.simple_hash(13, 12, 8, items, mx - 1)
    assert rc == oracle_mod.E_BIN_OVERFLOW and mx2 == mx


def test_pbh_same_bin_and_low_bits_means_same_image(oracle_mod):
    # Section 3.3: bin = x_H xor H(x_L); equal x_L and equal bin under the
    # same hash function force equal x_H.  Exhaust a small domain.
    seen = {}
    for x in range(20000):
        xl, bins = oracle_mod.hash_item(3, 6, 4, x)
        for i, b in enumerate(bins):
            key = (i, b, xl)
            h0 = (oracle_mod.mix64(x ^ oracle_mod.mix64(3 + 0x9E3779B97F4A7C15)) & (2**10 - 1))
            assert seen.setdefault(key, h0) == h0


def test_mu_values(oracle_mod):
    for row in golden("paper_values.json")["mu"]:
        assert oracle_mod.mu_bound(row["n"], row["b"]) == row["mu"]
    from scipy.stats import binom

    for n, b in [(1024, 4096), (1 << 16, 8192), (1 << 18, 8192)]:
        mu = oracle_mod.mu_bound(n, b)
        assert b * binom.sf(mu, 3 * n, 1 / b) <= 2**-40 < b * binom.sf(mu - 1, 3 * n, 1 / b)


# ------------------------------------------------------------- BFV (FV)
@pytest.fixture(scope="module")
def tiny(oracle_mod):
    c = oracle_mod.Ctx(N=16, t=T, prime_bits=[36, 36, 37], h=2, lambda_bar=6, hash_key=7, mu=4)
    s, rlk = c.keygen(3)
    return c, s, rlk


def rand_slots(rng, N):
    return rng.integers(0, T, N).astype(np.uint32)


def test_encrypt_decrypt(tiny):
    c, s, _ = tiny
    rng = np.random.default_rng(0)
    for seed in range(4):
        a = rand_slots(rng, c.N)
        sl, bud = c.decrypt(s, c.encrypt(s, c.encode(a), seed)[0])
        assert (sl == a).all() and bud > 50


def test_fresh_ciphertext_structure(tiny):
    # c0 + c1*s = round(Q*m/t) + e with |e| <= 21 (centred binomial, eta=21)
    c, s, _ = tiny
    m = c.encode(np.arange(c.N, dtype=np.uint32))
    ct = c.encrypt(s, m, 11)[0]
    Q = c.Q
    for n in range(c.N):
        c0 = int(sympy_crt(c.q, [int(ct[0, p, n]) for p in range(c.k)])[0])
        acc = c0
        c1 = [int(sympy_crt(c.q, [int(ct[1, p, j]) for p in range(c.k)])[0]) for j in range(c.N)]
        for j in range(c.N):  # (c1 * s)[n], negacyclic
            i = n - j
            sgn = 1
            if i < 0:
                i += c.N
                sgn = -1
            acc += sgn * c1[j] * int(s[i])
        e = (acc - (Q * int(m[n]) + (T - 1) // 2) // T) % Q
        e = e - Q if e > Q // 2 else e
        assert abs(e) <= 21


def test_plain_mult_add_scalar_const(tiny):
    c, s, _ = tiny
    rng = np.random.default_rng(1)
    a, p = rand_slots(rng, c.N), rand_slots(rng, c.N)
    ca = c.encrypt(s, c.encode(a), 1)[0]
    sl, _ = c.decrypt(s, c.ct_mul_pt(ca, c.encode(p)))
    assert (sl == (a.astype(np.int64) * p % T)).all()
    sl, _ = c.decrypt(s, c.ct_axpy(ca, -3, ca))
    assert (sl == (a.astype(np.int64) * -2 % T)).all()
    sl, _ = c.decrypt(s, c.ct_add_const(ca, -1))
    assert (sl == (a.astype(np.int64) - 1) % T).all()


def decrypt3(c, s, ct3):
    """Big-integer decryption of a 3-component ciphertext (d0 + d1 s + d2 s^2)."""
    N, Q = c.N, c.Q
    comps = [[int(sympy_crt(c.q, [int(ct3[comp, p, n]) for p in range(c.k)])[0]) for n in range(N)] for comp in range(3)]
    sl = [int(x) for x in s]
    s2 = negacyclic_schoolbook(sl, sl, N)
    z = [comps[0][n] for n in range(N)]
    t1 = negacyclic_schoolbook(comps[1], sl, N)
    t2 = negacyclic_schoolbook(comps[2], s2, N)
    z = [(z[n] + t1[n] + t2[n]) % Q for n in range(N)]
    z = [x - Q if x > Q // 2 else x for x in z]
    m = [((T * x + (Q - 1) // 2) // Q) % T for x in z]
    return c.decode(np.array(m, np.uint32))


def test_mult_decrypts_to_product_and_relin_preserves_it(tiny):
    c, s, rlk = tiny
    rng = np.random.default_rng(2)
    a, b = rand_slots(rng, c.N), rand_slots(rng, c.N)
    ca, cb = c.encrypt(s, c.encode(a), 1)[0], c.encrypt(s, c.encode(b), 2)[0]
    m3 = c.ct_mult(ca, cb)
    want = a.astype(np.int64) * b % T
    assert (decrypt3(c, s, m3) == want).all()
    r = c.relin(rlk, m3)
    sl, bud = c.decrypt(s, r)
    assert (sl == want).all() and bud > 0


def test_mult_words_against_big_integer_schoolbook(oracle_mod):
    # textbook FV: round(t/Q * (a~ (x) b~)) with centred lifts, exact integers
    c = oracle_mod.Ctx(N=8, t=T, prime_bits=[36, 37], h=1, lambda_bar=3)
    s, _ = c.keygen(5)
    rng = np.random.default_rng(6)
    ca = c.encrypt(s, c.encode(rand_slots(rng, 8)), 1)[0]
    cb = c.encrypt(s, c.encode(rand_slots(rng, 8)), 2)[0]
    Q, N = c.Q, c.N

    def lift(ct, comp):
        v = [int(sympy_crt(c.q, [int(ct[comp, p, n]) for p in range(c.k)])[0]) for n in range(N)]
        return [x - Q if x > Q // 2 else x for x in v]

    a0, a1, b0, b1 = lift(ca, 0), lift(ca, 1), lift(cb, 0), lift(cb, 1)
    x0 = negacyclic_schoolbook(a0, b0, N)
    x1 = [u + v for u, v in zip(negacyclic_schoolbook(a0, b1, N), negacyclic_schoolbook(a1, b0, N))]
    x2 = negacyclic_schoolbook(a1, b1, N)
    got = c.ct_mult(ca, cb)
    for comp, x in enumerate((x0, x1, x2)):
        for n in range(N):
            y = (T * x[n] + (Q - 1) // 2) // Q  # floor; Q odd -> round
            for p, q in enumerate(c.q):
                assert int(got[comp, p, n]) == y % q


def test_relin_key_structure(tiny):
    # rlk_i[0] + a_i s = e_i + g_i s^2 with g_i = 1 mod q_i, 0 mod q_j (j != i)
    c, s, rlk = tiny
    sl = [int(x) for x in s]
    s2 = negacyclic_schoolbook(sl, sl, c.N)
    for i in range(c.k):
        for j, q in enumerate(c.q):
            a = [int(x) for x in rlk[i, 1, j]]
            As = negacyclic_schoolbook(a, sl, c.N, q)
            for n in range(c.N):
                e = (int(rlk[i, 0, j, n]) + As[n] - (s2[n] if i == j else 0)) % q
                e = e - q if e > q // 2 else e
                assert abs(e) <= 21


def test_noise_budget_is_exact_threshold(tiny):
    # budget > 0 exactly when every coefficient's error is below Q/(2t)
    c, s, _ = tiny
    m = c.encode(np.zeros(c.N, np.uint32))
    ct = c.encrypt(s, m, 3)[0]
    _, b0 = c.decrypt(s, ct)
    ct2 = ct.copy()
    # add a large known error e* to c0[0]: |t*e*| close to Q/2 makes the budget ~0
    big = c.Q // (2 * T) - 10**6
    for p, q in enumerate(c.q):
        ct2[0, p, 0] = (int(ct2[0, p, 0]) + big) % q
    _, b1 = c.decrypt(s, ct2)
    assert b0 > b1 > -1 and b1 < 1


# --------------------------------------------------------------- PEPSI
def eq_truth_table_case(oracle_mod, h, lb, ell, N, bits, n_pairs, seed):
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=bits, h=h, ell=ell, lambda_bar=lb, mu=1)
    s, rlk = c.keygen(seed)
    rng = np.random.default_rng(seed)
    total = math.comb(ell, h)
    pairs = [(x, x) for x in range(min(total, n_pairs // 2))]
    while len(pairs) < n_pairs:
        pairs.append((int(rng.integers(total)), int(rng.integers(total))))
    for off in range(0, len(pairs), N):
        chunk = pairs[off:off + N]
        cl = np.full(N, oracle_mod.DUMMY, np.uint64)
        sv = np.full((1, N), oracle_mod.DUMMY, np.uint64)
        for i, (x, y) in enumerate(chunk):
            cl[i], sv[0, i] = x, y
        cts = c.encrypt(s, c.query_plaintexts(cl), seed + off)
        out = c.eval(rlk, cts, sv)
        slots, bud = c.decrypt(s, out)
        assert bud > 0
        for i, (x, y) in enumerate(chunk):
            assert int(slots[i]) == int(x == y), (h, x, y)
        assert (slots[len(chunk):] == 0).all()  # dummy vs dummy is 0


def test_arith_cw_eq_exhaustive_h2(oracle_mod):
    # all 15 x 15 pairs of CW(6, 2)
    c = oracle_mod.Ctx(N=64, t=T, prime_bits=[36, 36, 37], h=2, ell=6, lambda_bar=3, mu=1)
    s, rlk = c.keygen(1)
    words = list(range(15))
    pairs = [(x, y) for x in words for y in words]
    for off in range(0, len(pairs), 64):
        chunk = pairs[off:off + 64]
        cl = np.full(64, oracle_mod.DUMMY, np.uint64)
        sv = np.full((1, 64), oracle_mod.DUMMY, np.uint64)
        for i, (x, y) in enumerate(chunk):
            cl[i], sv[0, i] = x, y
        out = c.eval(rlk, c.encrypt(s, c.query_plaintexts(cl), off), sv)
        slots, bud = c.decrypt(s, out)
        assert bud > 0
        assert [int(v) for v in slots[: len(chunk)]] == [int(x == y) for x, y in chunk]


@pytest.mark.parametrize("h,lb,ell,bits", [(1, 4, 16, [36, 37]), (4, 6, 10, [55, 55, 54, 54]),
                                           (8, 8, 14, [55] * 6 + [54] * 2)])
def test_arith_cw_eq_truth_table(oracle_mod, h, lb, ell, bits):
    eq_truth_table_case(oracle_mod, h, lb, ell, 64, bits, 64, seed=h)


@pytest.mark.parametrize("h,bits,lb", [(2, [36, 36, 37], 10), (4, [55, 55, 54, 54], 12), (8, [55] * 6 + [54] * 2, 14)])
def test_psi_matches_brute_force(oracle_mod, h, bits, lb):
    from paper_2310_14565_gb300.workload import make_sets

    N = 64
    sets = make_sets(24, 150, 7, bits=32, seed_items=h, seed_plant=h + 1)
    load = oracle_mod.simple_hash(99, lb, 6, sets.server, 1000)[2]
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=bits, h=h, lambda_bar=lb, hash_key=99, mu=max(16, load))
    s, rlk = c.keygen(3)
    rc, Ts, _ = c.server_table(sets.server)
    assert rc == 0
    rc, cts, where = c.query(s, sets.client, 4)
    assert rc == 0
    out = c.eval(rlk, cts, Ts)
    assert c.last_counts == (c.ell * c.mu, c.mu * int(math.log2(h)))  # Thm 1 with log2 h products
    slots, bud = c.decrypt(s, out)
    assert bud > 0
    server = set(int(x) for x in sets.server)
    want = np.zeros(N, np.uint32)
    for u, x in enumerate(sets.client):
        want[where[u]] = int(int(x) in server)
    # hashed-domain intersection: same x_L in a bin the server item maps to
    hashed = np.zeros(N, np.uint32)
    srv = {}
    for y in sets.server:
        yl, bins = oracle_mod.hash_item(99, lb, 6, y)
        for b in bins:
            srv.setdefault(b, set()).add(yl)
    for u, x in enumerate(sets.client):
        xl, _ = oracle_mod.hash_item(99, lb, 6, x)
        hashed[where[u]] = int(xl in srv.get(int(where[u]), set()))
    assert (slots == hashed).all()
    assert (slots == want).all()
    out_c = c.eval(rlk, cts, Ts, mode=1, mask_seed=5)
    slots_c, _ = c.decrypt(s, out_c)
    assert int(slots_c.astype(np.int64).sum()) % T == len(sets.planted)
    assert not (slots_c == want).all()  # masked: individual slots hide the indicator


# ------------------------------------------------- deferred (lazy) rounding
def test_mult_sum_words_against_big_integer_schoolbook(oracle_mod):
    # one rounding of a sum of products: round(t/Q * sum_i a~_i (x) b~_i),
    # exact integers, centred lifts
    c = oracle_mod.Ctx(N=8, t=T, prime_bits=[36, 37], h=1, lambda_bar=3)
    s, _ = c.keygen(5)
    rng = np.random.default_rng(7)
    n = 3
    ca = np.stack([c.encrypt(s, c.encode(rand_slots(rng, 8)), 10 + i)[0] for i in range(n)])
    cb = np.stack([c.encrypt(s, c.encode(rand_slots(rng, 8)), 20 + i)[0] for i in range(n)])
    Q, N = c.Q, c.N

    def lift(ct, comp):
        v = [int(sympy_crt(c.q, [int(ct[comp, p, m]) for p in range(c.k)])[0]) for m in range(N)]
        return [x - Q if x > Q // 2 else x for x in v]

    X = [[0] * N for _ in range(3)]
    for i in range(n):
        a0, a1, b0, b1 = lift(ca[i], 0), lift(ca[i], 1), lift(cb[i], 0), lift(cb[i], 1)
        terms = (negacyclic_schoolbook(a0, b0, N),
                 [u + v for u, v in zip(negacyclic_schoolbook(a0, b1, N), negacyclic_schoolbook(a1, b0, N))],
                 negacyclic_schoolbook(a1, b1, N))
        for comp in range(3):
            X[comp] = [u + v for u, v in zip(X[comp], terms[comp])]
    got = c.ct_mult_sum(ca, cb)
    for comp in range(3):
        for m in range(N):
            y = (T * X[comp][m] + (Q - 1) // 2) // Q
            for p, q in enumerate(c.q):
                assert int(got[comp, p, m]) == y % q
    # a single product is the ordinary multiplication
    assert np.array_equal(c.ct_mult_sum(ca[:1], cb[:1]), c.ct_mult(ca[0], cb[0]))


def _lazy_case(oracle_mod, h, bits, lb):
    from paper_2310_14565_gb300.workload import make_sets

    N = 64
    sets = make_sets(24, 150, 7, bits=32, seed_items=h, seed_plant=h + 1)
    load = oracle_mod.simple_hash(99, lb, 6, sets.server, 1000)[2]
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=bits, h=h, lambda_bar=lb, hash_key=99, mu=max(7, load))
    s, rlk = c.keygen(3)
    rc, Ts, _ = c.server_table(sets.server)
    assert rc == 0
    rc, cts, where = c.query(s, sets.client, 4)
    assert rc == 0
    return c, s, rlk, sets, Ts, cts, where


@pytest.mark.parametrize("h,bits,lb", [(2, [36, 36, 37], 10), (4, [55, 55, 54, 54], 12), (8, [55] * 6 + [54] * 2, 14)])
def test_lazy_rescale_bounded_rounding_difference(oracle_mod, h, bits, lb):
    # Sum_l round(y_l) and round(Sum_l y_l) differ by at most (G + 1)/2 per
    # run of G layers, so the layer sums before relinearisation differ by at
    # most (nl + runs)/2 per coefficient; a one-layer run is the canonical
    # rounding itself
    c, s, rlk, sets, Ts, cts, where = _lazy_case(oracle_mod, h, bits, lb)
    mu = Ts.shape[0]
    out1, A1 = c.eval(rlk, cts, Ts, acc=True)
    for group in (2, 3, mu):
        outg, Ag = c.eval(rlk, cts, Ts, group=group, acc=True)
        runs = -(-mu // group)
        bound = (mu + runs) // 2
        for comp in range(3):
            for m in range(c.N):
                d = int(sympy_crt(c.q, [(int(Ag[comp, p, m]) - int(A1[comp, p, m])) % q
                                        for p, q in enumerate(c.q)])[0])
                d = d - c.Q if d > c.Q // 2 else d
                assert abs(d) <= bound
        assert not np.array_equal(Ag, A1)  # the words do change
    o1 = c.eval(rlk, cts, Ts, layer0=2, nlayers=1)
    assert np.array_equal(c.eval(rlk, cts, Ts, layer0=2, nlayers=1, group=4), o1)


@pytest.mark.parametrize("h,bits,lb", [(2, [36, 36, 37], 10), (4, [55, 55, 54, 54], 12), (8, [55] * 6 + [54] * 2, 14)])
def test_lazy_rescale_psi_matches_hashed_brute_force(oracle_mod, h, bits, lb):
    c, s, rlk, sets, Ts, cts, where = _lazy_case(oracle_mod, h, bits, lb)
    mu = Ts.shape[0]
    srv = {}
    for y in sets.server:
        yl, bins = oracle_mod.hash_item(99, lb, 6, y)
        for b in bins:
            srv.setdefault(b, set()).add(yl)
    hashed = np.zeros(c.N, np.uint32)
    for u, x in enumerate(sets.client):
        xl, _ = oracle_mod.hash_item(99, lb, 6, x)
        hashed[where[u]] = int(xl in srv.get(int(where[u]), set()))
    budgets = []
    for group in (3, mu):
        slots, bud = c.decrypt(s, c.eval(rlk, cts, Ts, group=group))
        assert bud > 0 and (slots == hashed).all()
        budgets.append(bud)
        slots_c, _ = c.decrypt(s, c.eval(rlk, cts, Ts, mode=1, mask_seed=5, group=group))
        assert int(slots_c.astype(np.int64).sum()) % T == int(hashed.sum())
    _, b1 = c.decrypt(s, c.eval(rlk, cts, Ts))
    assert budgets[-1] >= b1 - 1.0  # fewer roundings: no worse noise


# ------------------------------------------- labelled PSI and PSI-Sum
def test_mult_sum_with_values_against_big_integer_schoolbook(oracle_mod):
    # round(t/Q * sum_i v~_i (x) a~_i (x) b~_i), v~ the centred lift of a
    # plaintext, exact integers
    c = oracle_mod.Ctx(N=8, t=T, prime_bits=[36, 37], h=1, lambda_bar=3)
    s, _ = c.keygen(5)
    rng = np.random.default_rng(8)
    n = 2
    ca = np.stack([c.encrypt(s, c.encode(rand_slots(rng, 8)), 30 + i)[0] for i in range(n)])
    cb = np.stack([c.encrypt(s, c.encode(rand_slots(rng, 8)), 40 + i)[0] for i in range(n)])
    v = rng.integers(0, T, size=(n, 8)).astype(np.uint32)
    Q, N = c.Q, c.N

    def lift(ct, comp):
        w = [int(sympy_crt(c.q, [int(ct[comp, p, m]) for p in range(c.k)])[0]) for m in range(N)]
        return [x - Q if x > Q // 2 else x for x in w]

    X = [[0] * N for _ in range(3)]
    for i in range(n):
        a0, a1, b0, b1 = lift(ca[i], 0), lift(ca[i], 1), lift(cb[i], 0), lift(cb[i], 1)
        vi = [int(x) if x <= T // 2 else int(x) - T for x in v[i]]
        terms = (negacyclic_schoolbook(a0, b0, N),
                 [u + w for u, w in zip(negacyclic_schoolbook(a0, b1, N), negacyclic_schoolbook(a1, b0, N))],
                 negacyclic_schoolbook(a1, b1, N))
        for comp in range(3):
            X[comp] = [u + w for u, w in zip(X[comp], negacyclic_schoolbook(terms[comp], vi, N))]
    got = c.ct_mult_sum(ca, cb, v)
    for comp in range(3):
        for m in range(N):
            y = (T * X[comp][m] + (Q - 1) // 2) // Q
            for p, q in enumerate(c.q):
                assert int(got[comp, p, m]) == y % q


def test_value_table_brute_force(oracle_mod):
    from paper_2310_14565_gb300.workload import make_sets

    lb, logb = 6, 4
    items = make_sets(4, 90, 2, bits=32, seed_items=3, seed_plant=4).server
    values = (np.arange(len(items), dtype=np.uint32) * 7919 + 1) % T
    rc, Tt, V, load = oracle_mod.simple_hash_values(7, lb, logb, items, values, 40)
    assert rc == 0
    rc2, T2, _ = oracle_mod.simple_hash(7, lb, logb, items, 40)
    assert np.array_equal(Tt, T2)
    hashed = [oracle_mod.hash_item(7, lb, logb, int(x)) for x in items]
    for layer in range(Tt.shape[0]):
        for b in range(1 << logb):
            if Tt[layer, b] == oracle_mod.DUMMY:
                assert V[layer, b] == 0
                continue
            # the first item (input order) with this x_L among those mapping to bin b
            owner = next(u for u, (xl, bins) in enumerate(hashed) if xl == int(Tt[layer, b]) and b in bins)
            assert V[layer, b] == values[owner]


def _valued_case(oracle_mod, h, bits, lb, seed):
    from paper_2310_14565_gb300.workload import make_sets

    N = 64
    sets = make_sets(24, 150, 7, bits=32, seed_items=seed, seed_plant=seed + 1)
    values = np.random.default_rng(seed).integers(1, T, size=150).astype(np.uint32)
    load = oracle_mod.simple_hash(99, lb, 6, sets.server, 1000)[2]
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=bits, h=h, lambda_bar=lb, hash_key=99, mu=max(7, load))
    s, rlk = c.keygen(3)
    rc, Ts, V, _ = c.server_table_values(sets.server, values)
    assert rc == 0
    rc, cts, where = c.query(s, sets.client, 4)
    assert rc == 0
    # expected label per client slot: the value stored with the matching x_L in its bin (hashed domain)
    labels = np.zeros(N, np.uint32)
    for u, x in enumerate(sets.client):
        xl, _ = oracle_mod.hash_item(99, lb, 6, x)
        col = Ts[:, where[u]]
        hit = np.nonzero(col == xl)[0]
        if hit.size:
            labels[where[u]] = V[hit[0], where[u]]
    return c, s, rlk, sets, Ts, V, cts, where, labels


@pytest.mark.parametrize("h,bits,lb", [(1, [36, 37], 8), (2, [36, 36, 37], 10), (4, [55, 55, 54, 54], 12),
                                       (8, [55] * 6 + [54] * 2, 14)])
def test_labelled_psi_and_psi_sum(oracle_mod, h, bits, lb):
    c, s, rlk, sets, Ts, V, cts, where, labels = _valued_case(oracle_mod, h, bits, lb, seed=h + 20)
    assert int((labels != 0).sum()) >= len(sets.planted)
    for group in (1, Ts.shape[0]):
        out = c.eval(rlk, cts, Ts, mode=2, V=V, group=group)
        slots, bud = c.decrypt(s, out)
        assert bud > 0 and np.array_equal(slots, labels), group  # Algorithm 4
        outs = c.eval(rlk, cts, Ts, mode=3, mask_seed=5, V=V, group=group)
        ss, bud = c.decrypt(s, outs)
        assert bud > 0
        assert int(ss.astype(np.int64).sum()) % T == int(labels.astype(np.int64).sum()) % T  # Algorithm 5
        assert not np.array_equal(ss, labels)  # masked
    # values all 1: the labelled result is the indicator
    ones = (V != 0).astype(np.uint32)
    ind = c.decrypt(s, c.eval(rlk, cts, Ts))[0]
    assert np.array_equal(c.decrypt(s, c.eval(rlk, cts, Ts, mode=2, V=ones))[0], ind)


# ------------------------------------------- response modulus switching
def test_mod_switch_words_against_big_integers(oracle_mod):
    # round(c~ * Q_r / Q) of the centred lift, exact integers
    c = oracle_mod.Ctx(N=8, t=T, prime_bits=[36, 36, 37], h=1, lambda_bar=3)
    s, _ = c.keygen(5)
    rng = np.random.default_rng(9)
    ct = c.encrypt(s, c.encode(rand_slots(rng, 8)), 3)[0]
    Q = c.Q
    for r in (1, 2, 3):
        Qr = math.prod(c.q[:r])
        got = c.mod_switch(ct, r)
        for comp in range(2):
            for m in range(8):
                x = int(sympy_crt(c.q, [int(ct[comp, p, m]) for p in range(c.k)])[0])
                x = x - Q if x > Q // 2 else x
                num = x * Qr
                y = (2 * num + Q) // (2 * Q)  # round(num / Q), Q odd: no ties
                for p in range(r):
                    assert int(got[comp, p, m]) == y % c.q[p]
    assert np.array_equal(c.mod_switch(ct, 3), ct)


@pytest.mark.parametrize("bits", [[36, 36, 37], [55, 55, 54, 54]])
def test_mod_switch_preserves_decryption(oracle_mod, bits):
    c = oracle_mod.Ctx(N=64, t=T, prime_bits=bits, h=1, lambda_bar=6)
    s, rlk = c.keygen(2)
    rng = np.random.default_rng(10)
    a, b = rand_slots(rng, 64), rand_slots(rng, 64)
    cts = c.encrypt(s, np.stack([c.encode(a), c.encode(b)]), 4)
    prod = c.relin(rlk, c.ct_mult(cts[0], cts[1]))  # a noisier ciphertext too
    want = a.astype(np.int64) * b % T
    for ct, slots in ((cts[0], a), (prod, want)):
        full, b_full = c.decrypt(s, ct)
        for r in range(1, c.k + 1):
            sw = c.mod_switch(ct, r)
            got, bud = c.decrypt(s, sw)
            assert bud > 0 and np.array_equal(got, slots) and np.array_equal(got, full)
            # c' = c Q_r / Q + eps with |eps| <= 1/2 per coefficient, so
            # |[t z']_{Q_r}| <= |[t z]_Q| Q_r / Q + t (1 + |s|_1) / 2
            lq, lqr = math.log2(c.Q), sum(math.log2(q) for q in c.q[:r])
            e_full = 2.0 ** (lq - 1 - b_full)
            bound = lqr - 1 - math.log2(e_full * 2.0 ** (lqr - lq) + T * (1 + int(np.abs(s).sum())) / 2)
            assert bud >= bound - 1e-6 or r == c.k


@pytest.mark.parametrize("h,bits,lb", [(4, [55, 55, 54, 54], 12), (8, [55] * 6 + [54] * 2, 14)])
def test_psi_response_switched_to_one_prime(oracle_mod, h, bits, lb):
    c, s, rlk, sets, Ts, cts, where = _lazy_case(oracle_mod, h, bits, lb)
    out = c.eval(rlk, cts, Ts)
    full, _ = c.decrypt(s, out)
    for r in (1, 2):
        slots, bud = c.decrypt(s, c.mod_switch(out, r))
        assert bud > 0 and np.array_equal(slots, full)


# ----------------------------------------------- more bins than slots
def test_psi_with_more_bins_than_slots(oracle_mod):
    # b = 4N bins: four blocks of N slots, each evaluated against its own
    # block of the server table; the blocks' slots together equal the
    # hashed-domain brute force over all b bins
    from paper_2310_14565_gb300.workload import make_sets

    N, B, lb = 64, 4, 10
    sets = make_sets(150, 300, 9, bits=32, seed_items=61, seed_plant=62)
    load = oracle_mod.simple_hash(99, lb, 8, sets.server, 1000)[2]
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=[55, 55, 54, 54], h=4, lambda_bar=lb, hash_key=99, mu=max(5, load),
                       bins=N * B)
    s, rlk = c.keygen(3)
    rc, Ts, _ = c.server_table(sets.server)
    assert rc == 0 and Ts.shape == (c.mu, N * B)
    rc, cts, where = c.query(s, sets.client, 4)
    assert rc == 0 and cts.shape == (B, c.ell, 2, c.k, N)
    slots = np.concatenate([c.decrypt(s, c.eval(rlk, cts[b], Ts[:, b * N:(b + 1) * N]))[0] for b in range(B)])
    srv = {}
    for y in sets.server:
        yl, bins = oracle_mod.hash_item(99, lb, 8, y)
        for bb in bins:
            srv.setdefault(bb, set()).add(yl)
    want = np.zeros(N * B, np.uint32)
    for u, x in enumerate(sets.client):
        xl, _ = oracle_mod.hash_item(99, lb, 8, x)
        want[where[u]] = int(xl in srv.get(int(where[u]), set()))
    assert np.array_equal(slots, want) and int(want.sum()) >= 9
    # more client items than one block holds
    assert len(sets.client) > N


def test_psi_with_client_bins_of_two_slots(oracle_mod):
    """gamma = 2: 100 client items in 64 bins (cuckoo with one slot per bin
    cannot hold them).  The request is two batches of ell ciphertexts (batch
    i: slot i of every bin); Algorithm 2 returns one indicator ciphertext per
    batch; together their slots equal the hashed-domain brute force for every
    client item, at where[u] = bin * 2 + slot.  Cardinality: the two masked
    responses' slots sum to the intersection size."""
    from paper_2310_14565_gb300.workload import make_sets

    N, g, lb = 64, 2, 10
    sets = make_sets(100, 200, 8, bits=32, seed_items=71, seed_plant=72)
    load = oracle_mod.simple_hash(99, lb, 6, sets.server, 1000)[2]
    c = oracle_mod.Ctx(N=N, t=T, prime_bits=[55, 55, 54, 54], h=4, lambda_bar=lb, hash_key=99, mu=max(5, load),
                       gamma=g)
    s, rlk = c.keygen(3)
    rc, Ts, _ = c.server_table(sets.server)
    assert rc == 0
    assert oracle_mod.cuckoo(99, lb, 6, sets.client)[0] == oracle_mod.E_CUCKOO_FAIL
    rc, cts, where = c.query(s, sets.client, 4)
    assert rc == 0 and cts.shape == (g, c.ell, 2, c.k, N)
    res = [c.decrypt(s, c.eval(rlk, cts[i], Ts)) for i in range(g)]
    assert all(b > 0 for _, b in res)
    got = np.stack([sl for sl, _ in res], axis=1).reshape(-1)  # [bin][slot]
    srv = {}
    for y in sets.server:
        yl, bins = oracle_mod.hash_item(99, lb, 6, y)
        for bb in bins:
            srv.setdefault(bb, set()).add(yl)
    want = np.zeros(N * g, np.uint32)
    for u, x in enumerate(sets.client):
        xl, _ = oracle_mod.hash_item(99, lb, 6, x)
        want[where[u]] = int(xl in srv.get(int(where[u]) // g, set()))
    assert np.array_equal(got, want) and int(want.sum()) >= 8
    card = sum(int(c.decrypt(s, c.eval(rlk, cts[i], Ts, mode=1, mask_seed=5 + i))[0].astype(np.int64).sum())
               for i in range(g))
    assert card % T == int(want.sum())


# ------------------------------------------- false matches (Lemma 1)
def test_false_match_rate_follows_the_hashed_collision_model(oracle_mod):
    # A client item outside the server set matches when a server item of
    # its bin has the same lambda_bar-bit x_L.  Permutation-based hashing
    # puts log2 b of the lambda hash bits into the bin, so inside a bin the
    # x_L of two unrelated items agree with probability 2^-lambda_bar.  Over
    # seeded trials the false-match count must follow
    # E = sum over non-member client items of (distinct x_L stored in its
    # bin) / 2^lambda_bar, within Poisson noise (4 sigma), and be nonzero.
    from paper_2310_14565_gb300.workload import make_sets

    lb, logb, m, n, trials = 6, 6, 40, 60, 150
    measured, expected = 0, 0.0
    for tr in range(trials):
        sets = make_sets(m, n, 5, bits=32, seed_items=500 + tr, seed_plant=900 + tr)
        rc, table, where = oracle_mod.cuckoo(7 + tr, lb, logb, sets.client)
        assert rc == 0
        rc, Ts, _ = oracle_mod.simple_hash(7 + tr, lb, logb, sets.server, 200)
        assert rc == 0
        server = set(int(y) for y in sets.server)
        for u, x in enumerate(sets.client):
            if int(x) in server:
                continue
            col = Ts[:, where[u]]
            stored = col[col != oracle_mod.DUMMY]
            expected += len(set(int(v) for v in stored)) / 2.0 ** lb
            measured += int(int(table[where[u]]) in set(int(v) for v in stored))
    assert measured > 0
    assert abs(measured - expected) <= 4 * math.sqrt(expected) + 1, (measured, expected)


def test_relin_words_against_big_integer_schoolbook(oracle_mod):
    # RNS-digit key switching without a special prime: d_i = [d2]_{q_i} in
    # [0, q_i), (c0, c1) += sum_i d_i * rlk_i, products in Z_{q_j}[X]/(X^N+1)
    # recomputed with Python integers
    c = oracle_mod.Ctx(N=8, t=T, prime_bits=[36, 36, 37], h=1, lambda_bar=3)
    s, rlk = c.keygen(9)
    rng = np.random.default_rng(11)
    ct3 = np.stack([np.stack([rng.integers(0, q, size=8, dtype=np.uint64) for q in c.q]) for _ in range(3)])
    got = c.relin(rlk, ct3)
    N = c.N
    for comp in range(2):
        for j, qj in enumerate(c.q):
            acc = [int(x) for x in ct3[comp, j]]
            for i in range(c.k):
                digit = [int(x) % qj for x in ct3[2, i]]  # [d2]_{q_i}, then taken mod q_j
                prod = negacyclic_schoolbook(digit, [int(x) for x in rlk[i, comp, j]], N, qj)
                acc = [(a + b) % qj for a, b in zip(acc, prod)]
            assert [int(x) for x in got[comp, j]] == acc
