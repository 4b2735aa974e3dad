"""The bounds the device arithmetic relies on, checked with Python integers
for every prime size the library accepts (ciphertext primes of 20..60 bits,
59- and 61-bit auxiliary primes, t = 65537):

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
  mod 2^64 even where SM wraps;
- the forward transforms of primes below 2^59, whose butterflies do not
  reduce their sum input: below (4 + 2 log2 N) q < 2^64 at every stage, and
  the residues of the reducing form after one Barrett reduction;
- Shoup's product in 32-bit words for the plaintext modulus, with the
  companion taken from the upper half of the 64-bit one."""
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


def ntt_prime_below(bits, logn):
    """The largest prime below 2^bits that is 1 mod 2N (N = 2^logn)."""
    step = 2 << logn
    q = ((1 << bits) - 1) // step * step + 1
    while not is_prime(q):
        q -= step
    return q


def brev(i, bits):
    return int(format(i, "0%db" % bits)[::-1], 2)


def forward_lazy(x, q, logn, grow):
    """Negacyclic Cooley-Tukey transform of x (values in [0, 4q)), natural
    order in, bit-reversed order out, in the stage and twiddle order of the
    library's fused forward transforms: stage s pairs elements N/2^(s+1)
    apart, block i of the stage takes the twiddle psi^brev(2^s + i).  Each
    butterfly is (u + T, u + 2q - T), T = w x mod q lazily by Shoup in
    [0, 2q); without grow, u is first reduced below 2q.  Returns the reduced
    output and the largest value any stage held."""
    n = 1 << logn
    n2 = 2 * n
    psi = next(p for p in (pow(g, (q - 1) // n2, q) for g in range(2, 200)) if pow(p, n, q) == q - 1)
    tw = [pow(psi, brev(i, logn), q) for i in range(n)]
    x = list(x)
    peak = max(x)
    for s in range(logn):
        m, t = 1 << s, n >> (s + 1)
        for i in range(m):
            w = tw[m + i]
            ws = (w << 64) // q
            for j in range(2 * i * t, 2 * i * t + t):
                u = x[j]
                if not grow and u >= 2 * q:
                    u -= 2 * q
                v = shoup_lazy(x[j + t], w, ws, q)
                assert v < 2 * q
                x[j], x[j + t] = u + v, u + 2 * q - v
        peak = max(peak, max(x))
    out = []
    m64 = (1 << 64) // q
    for v in x:
        assert v < (1 << 64)
        if grow:  # one-word Barrett: [0, 2^64) -> [0, 2q) -> [0, q)
            v -= ((v * m64) >> 64) * q
            assert v < 2 * q
        elif v >= 2 * q:
            v -= 2 * q
        out.append(v - q if v >= q else v)
    return out, peak, psi


@pytest.mark.parametrize("logn", [12, 13, 14])
def test_growing_forward_transform_fits_64_bits_below_2_59(logn):
    """The forward transforms of primes below 2^59 skip the reduction of the
    butterfly's sum input: each stage adds less than 2q, so from inputs in
    [0, 4q) the values stay below (4 + 2 log2 N) q <= 32 q < 2^64, and one
    Barrett reduction at the store gives the residues of the reducing form.
    Checked at the largest NTT-friendly prime below 2^59 on the largest
    inputs the transform accepts and on random ones; the outputs are the
    evaluations at psi^(2 brev(k) + 1)."""
    q = ntt_prime_below(59, logn)
    assert q < (1 << 59) and (4 + 2 * logn) * q < (1 << 64)
    n = 1 << logn
    rng = random.Random(logn)
    for x in ([4 * q - 1] * n, [rng.randrange(4 * q) for _ in range(n)]):
        grow, peak, psi = forward_lazy(x, q, logn, True)
        plain, peak_plain, _ = forward_lazy(x, q, logn, False)
        assert peak < (4 + 2 * logn) * q
        assert peak_plain < 4 * q
        assert grow == plain
        for k in (0, 1, n // 2 + 3, n - 1):
            z = pow(psi, 2 * brev(k, logn) + 1, q)
            assert grow[k] == sum(v * pow(z, i, q) for i, v in enumerate(x)) % q


@pytest.mark.parametrize("q", [65537, 786433, ntt_prime_below(30, 14)])
def test_32_bit_shoup_from_the_upper_half_of_the_64_bit_companion(q):
    """The plaintext-modulus transforms (q < 2^30) run in 32-bit words with
    the companion floor(w 2^32 / q) taken as the upper half of the 64-bit
    floor(w 2^64 / q): the two are equal, and x w - floor(x ws / 2^32) q mod
    2^32 lies in [0, 2q) and is x w mod q for every x < 4q (the inverse
    butterfly's difference input; 4q < 2^32)."""
    rng = random.Random(q)
    M32 = (1 << 32) - 1
    for w in [1, q - 1, q // 2] + [rng.randrange(q) for _ in range(200)]:
        ws = ((w << 64) // q) >> 32
        assert ws == (w << 32) // q
        for x in [0, 4 * q - 1, 2 * q] + [rng.randrange(4 * q) for _ in range(50)]:
            r = (x * w - ((x * ws) >> 32) * q) & M32
            assert r < 2 * q and r % q == x * w % q
