"""The bounds the device arithmetic relies on, checked with Python integers
for every prime size the library accepts (ciphertext primes of 20..60 bits,
61-bit auxiliary primes, t = 65537):

- one-constant Barrett for a b mod q with a, b < 2^n: the quotient
  floor(floor(ab / 2^(n-1)) mu / 2^64), mu = floor(2^(n+63) / q), is short
  of floor(ab / q) by at most 2, and mu fits in 64 bits;
- one-word Barrett for x < 2^64: floor(x floor(2^64/q) / 2^64) is short by
  at most 1;
- a 128-bit value as hi (2^64 mod q) by Shoup plus lo by one-word Barrett:
  both parts below 2q, their sum below 2^64;
- the multiply-accumulate's Karatsuba partial sums over one fold interval
  (2^(63 - max(bits + 1, 2s)) terms) plus the residue a fold leaves: S0,
  S2 and the middle sum S1 each stay below 2^64, so S1 = SM - S0 - S2 holds
  mod 2^64 even where SM wraps."""
import random

import pytest

M64 = (1 << 64) - 1


def is_prime(n):
    """Miller-Rabin with the first twelve prime bases: deterministic below 3.3e24."""
    if n < 2:
        return False
    bases = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in bases:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d, r = d // 2, r + 1
    for a in bases:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def prevprime(n):
    n -= 1
    while not is_prime(n):
        n -= 1
    return n


def nextprime(n):
    n += 1
    while not is_prime(n):
        n += 1
    return n


def primes_of_sizes():
    qs = [65537]
    for bits in list(range(20, 62)):
        qs.append(prevprime(1 << bits))
        qs.append(nextprime(1 << (bits - 1)))
    return qs


def shoup_lazy(x, w, ws, q):
    return (x * w - ((x * ws) >> 64) * q) & M64


@pytest.mark.parametrize("q", primes_of_sizes())
def test_reductions_short_by_their_bound(q):
    n = q.bit_length()
    mu = (1 << (n + 63)) // q
    m64 = (1 << 64) // q
    c64 = (1 << 64) % q
    c64s = (c64 << 64) // q
    assert mu < (1 << 64)
    rng = random.Random(q)
    top = (1 << n) - 1
    cases = [(top, top), (top, top - 1), (q - 1, q - 1), (0, 0)]
    cases += [(rng.randrange(1 << n), rng.randrange(1 << n)) for _ in range(400)]
    for a, b in cases:
        x = a * b
        qhat = ((x >> (n - 1)) * mu) >> 64
        assert 0 <= x // q - qhat <= 2
        assert x - qhat * q < 3 * q < (1 << 63)
    for x in [M64, 0, q, min(q * q - 1, M64)] + [rng.randrange(1 << 64) for _ in range(400)]:
        qhat = (x * m64) >> 64
        assert 0 <= x // q - qhat <= 1
    for v in [(1 << 128) - 1, q * q, (q - 1) << 64] + [rng.randrange(1 << 128) for _ in range(400)]:
        hi, lo = v >> 64, v & M64
        a = shoup_lazy(hi, c64, c64s, q)
        b = (lo - ((lo * m64) >> 64) * q) & M64
        assert a < 2 * q and b < 2 * q and a + b < (1 << 64)
        assert (a + b) % q == v % q


@pytest.mark.parametrize("bits", list(range(20, 61)))
def test_karatsuba_sums_fit_over_a_fold(bits):
    q = prevprime(1 << bits)
    s = (bits + 1) // 2
    worst = max(bits + 1, 2 * s)
    terms = 1 << min(20, 63 - worst)  # the library's fold interval
    lo_max, hi_max = (1 << s) - 1, (q - 1) >> s  # split halves of values below q
    s0 = (q - 1) + terms * lo_max * lo_max  # a fold leaves a residue below q in S0
    s2 = terms * hi_max * hi_max
    s1 = terms * 2 * lo_max * hi_max
    assert max(s0, s1, s2) < (1 << 64)
    # the middle sum recovered mod 2^64 from a wrapped SM equals the true one
    rng = random.Random(bits)
    S0 = SM = rng.randrange(q)  # a fold restarts S0 and SM at the residue, S2 at 0
    S1 = S2 = 0
    for _ in range(terms if terms <= 256 else 256):
        x, c = rng.randrange(q), rng.randrange(q)
        xl, xh, cl, ch = x & lo_max, x >> s, c & lo_max, c >> s
        S0 += cl * xl
        S2 += ch * xh
        SM = (SM + (cl + ch) * (xl + xh)) & M64
        S1 += cl * xh + ch * xl
    assert (SM - S0 - S2) & M64 == S1
