"""Plain CPU oracle for PEPSI's server-side evaluation (arXiv 2310.14565).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the cpu_baseline / reference legs of ``bench.py``, never by the
product package.  It shares no code with the CUDA library; both sides only
take their inputs (item sets, seeds) from ``paper_2310_14565_gb300.workload``.

The arithmetic lives in ``pepsi_oracle.c`` (plain C, 128-bit ``%`` modular
products, schoolbook big integers).  This module compiles it with gcc on
first use and exposes thin numpy wrappers plus the parameter rules:

* Eq. 1 (code length), Section 4.1.
* the server bin bound mu: the paper's values for its own (n, b) pairs
  (Tables 5-7), otherwise the smallest mu with
  b * P[Binomial(3n, 1/b) > mu] <= 2^-40 (Section 7's 2^-40 target).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pepsi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DUMMY = np.uint64(0xFFFFFFFFFFFFFFFF)
OK, E_PARAM, E_BIN_OVERFLOW, E_CUCKOO_FAIL, E_NOMEM = 0, 1, 2, 3, 4

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP if available)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.or_is_prime.argtypes = [C.c_uint64]
        L.or_is_prime.restype = C.c_int
        L.or_mix64.argtypes = [C.c_uint64]
        L.or_mix64.restype = C.c_uint64
        L.or_draw.argtypes = [C.c_uint64] * 3
        L.or_draw.restype = C.c_uint64
        L.or_sample_mod.argtypes = [C.c_uint64] * 4
        L.or_sample_mod.restype = C.c_uint64
        L.or_sample_cbd.argtypes = [C.c_uint64] * 3
        L.or_sample_cbd.restype = C.c_int
        L.or_stream.argtypes = [C.c_uint64] * 3
        L.or_stream.restype = C.c_uint64
        L.or_find_prime.argtypes = [C.c_uint32, C.c_uint32, u64p, C.c_uint32]
        L.or_find_prime.restype = C.c_uint64
        L.or_min_root.argtypes = [C.c_uint64, C.c_uint32]
        L.or_min_root.restype = C.c_uint64
        L.or_ntt_direct.argtypes = [u64p, C.c_uint32, C.c_uint64, C.c_uint64, u64p]
        L.or_ntt_fwd.argtypes = [u64p, C.c_uint32, C.c_uint64, C.c_uint64]
        L.or_ntt_inv.argtypes = [u64p, C.c_uint32, C.c_uint64, C.c_uint64]
        L.or_crt.argtypes = [u64p, u64p, C.c_uint32, u32p, C.c_uint32]
        L.or_create.argtypes = [C.c_uint32, C.c_uint64, C.c_uint32, u8p]
        L.or_create.restype = C.c_void_p
        L.or_free.argtypes = [C.c_void_p]
        L.or_info.argtypes = [C.c_void_p, u64p, u64p, u64p, u32p, u64p]
        L.or_log2_q.argtypes = [C.c_void_p]
        L.or_log2_q.restype = C.c_double
        L.or_encode.argtypes = [C.c_void_p, u32p, u32p]
        L.or_decode.argtypes = [C.c_void_p, u32p, u32p]
        L.or_binom.argtypes = [C.c_uint64, C.c_uint64]
        L.or_binom.restype = C.c_uint64
        L.or_code_length.argtypes = [C.c_uint32, C.c_uint32]
        L.or_code_length.restype = C.c_uint32
        L.or_cw_encode.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, u16p]
        L.or_hash_item.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64,
                                   C.POINTER(C.c_uint64), u32p]
        L.or_cuckoo.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, u64p, C.c_uint32, u64p, i32p]
        L.or_cuckoo_g.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, u64p, C.c_uint32, u64p, i32p]
        L.or_simple_hash.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, u64p, C.c_uint64, C.c_uint32,
                                     u64p, C.POINTER(C.c_uint32)]
        L.or_keygen.argtypes = [C.c_void_p, C.c_uint64, i8p, u64p]
        L.or_encrypt.argtypes = [C.c_void_p, i8p, u32p, C.c_uint32, C.c_uint64, u64p]
        L.or_decrypt.argtypes = [C.c_void_p, i8p, u64p, u32p, C.POINTER(C.c_double)]
        L.or_decrypt_primes.argtypes = [C.c_void_p, i8p, u64p, C.c_uint32, u32p, C.POINTER(C.c_double)]
        L.or_mod_switch.argtypes = [C.c_void_p, u64p, C.c_uint32, u64p]
        L.or_pt_lift.argtypes = [C.c_void_p, u32p, u64p]
        L.or_ct_mul_pt.argtypes = [C.c_void_p, u64p, u32p, u64p]
        L.or_ct_axpy.argtypes = [C.c_void_p, u64p, C.c_int64, u64p, C.c_uint32, u64p]
        L.or_ct_scale.argtypes = [C.c_void_p, u64p, C.c_int64, C.c_uint32]
        L.or_ct_add_const.argtypes = [C.c_void_p, u64p, C.c_int64]
        L.or_ct_mult.argtypes = [C.c_void_p, u64p, u64p, u64p]
        L.or_relin.argtypes = [C.c_void_p, u64p, u64p, u64p]
        L.or_server_plaintext.argtypes = [C.c_void_p, u64p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, u64p]
        L.or_query_plaintexts.argtypes = [C.c_void_p, u64p, C.c_uint32, C.c_uint32, u32p]
        L.or_ct_mult_sum.argtypes = [C.c_void_p, u64p, u64p, C.c_void_p, C.c_uint32, u64p]
        L.or_simple_hash_values.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, u64p, u32p, C.c_uint64,
                                            C.c_uint32, u64p, u32p, C.POINTER(C.c_uint32)]
        L.or_eval.argtypes = [C.c_void_p, u64p, u64p, C.c_uint32, C.c_uint32, u64p, C.c_void_p, C.c_uint32,
                              C.c_uint32, C.c_uint32, C.c_int, C.c_uint64, C.c_uint32, u64p, C.c_void_p,
                              C.c_void_p, C.c_void_p, u64p]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_get_threads.restype = C.c_int
        _lib = L
    return _lib


# ---------------------------------------------------------------- scalars
def is_prime(n: int) -> bool:
    return bool(lib().or_is_prime(n))


def mix64(z: int) -> int:
    return lib().or_mix64(z & 0xFFFFFFFFFFFFFFFF)


def draw(seed, stream, idx) -> int:
    return lib().or_draw(seed, stream, idx)


def sample_mod(seed, stream, pos, bound) -> int:
    return lib().or_sample_mod(seed, stream, pos, bound)


def sample_cbd(seed, stream, pos) -> int:
    return lib().or_sample_cbd(seed, stream, pos)


def stream(purpose, index, prime) -> int:
    return lib().or_stream(purpose, index, prime)


def find_prime(bits: int, N: int, taken=()) -> int:
    tk = np.array(list(taken) or [0], dtype=np.uint64)
    return lib().or_find_prime(bits, N, tk, len(taken))


def min_root(q: int, N: int) -> int:
    return lib().or_min_root(q, N)


def ntt_direct(a, N, q, psi):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros(N, dtype=np.uint64)
    lib().or_ntt_direct(a, N, q, psi, out)
    return out


def ntt_fwd(a, N, q, psi):
    a = np.array(a, dtype=np.uint64)
    lib().or_ntt_fwd(a, N, q, psi)
    return a


def ntt_inv(a, N, q, psi):
    a = np.array(a, dtype=np.uint64)
    lib().or_ntt_inv(a, N, q, psi)
    return a


def crt(residues, primes) -> int:
    r = np.ascontiguousarray(residues, dtype=np.uint64)
    p = np.ascontiguousarray(primes, dtype=np.uint64)
    limbs = np.zeros(64, dtype=np.uint32)
    rc = lib().or_crt(r, p, len(p), limbs, 64)
    assert rc == 0
    return sum(int(x) << (32 * i) for i, x in enumerate(limbs))


def binom(n, r) -> int:
    return lib().or_binom(n, r)


def code_length(lambda_bar: int, h: int) -> int:
    """Eq. 1: smallest ell with C(ell, h) >= 2^lambda_bar."""
    return lib().or_code_length(lambda_bar, h)


def cw_encode(v: int, ell: int, h: int):
    pos = np.zeros(max(h, 1), dtype=np.uint16)
    rc = lib().or_cw_encode(v, ell, h, pos)
    if rc:
        raise ValueError("value out of range for CW(%d,%d)" % (ell, h))
    return [int(x) for x in pos[:h]]


def hash_item(hash_key, lambda_bar, logb, x):
    xl = C.c_uint64(0)
    bins = np.zeros(3, dtype=np.uint32)
    lib().or_hash_item(hash_key, lambda_bar, logb, int(x), C.byref(xl), bins)
    return int(xl.value), [int(b) for b in bins]


def cuckoo(hash_key, lambda_bar, logb, items, gamma=1):
    """Client cuckoo hashing into 2^logb bins of gamma slots: (rc, table
    [bin * gamma + slot] of x_L or DUMMY, where[u] = bin * gamma + slot)."""
    items = np.ascontiguousarray(items, dtype=np.uint64)
    table = np.zeros((1 << logb) * gamma, dtype=np.uint64)
    where = np.full(len(items), -1, dtype=np.int32)
    rc = lib().or_cuckoo_g(hash_key, lambda_bar, logb, gamma, items if len(items) else np.zeros(1, np.uint64),
                           len(items), table, where if len(items) else np.zeros(1, np.int32))
    return rc, table, where


def simple_hash(hash_key, lambda_bar, logb, items, mu):
    items = np.ascontiguousarray(items, dtype=np.uint64)
    T = np.zeros(mu * (1 << logb), dtype=np.uint64)
    mx = C.c_uint32(0)
    rc = lib().or_simple_hash(hash_key, lambda_bar, logb, items if len(items) else np.zeros(1, np.uint64),
                              len(items), mu, T, C.byref(mx))
    return rc, T.reshape(mu, 1 << logb), int(mx.value)


# ------------------------------------------------------------ parameters
PAPER_MU = {  # (n, b) -> mu, Tables 5, 6 and 7
    (1 << 20, 8192): 526, (1 << 24, 8192): 6710, (1 << 28, 8192): 100565,
    (1 << 18, 16384): 100, (1 << 20, 16384): 296, (1 << 22, 16384): 976,
    (1 << 24, 16384): 3487, (1 << 28, 16384): 50812,
}


def simple_hash_values(hash_key, lambda_bar, logb, items, values, mu):
    """Server table plus the value of the item stored at each (layer, bin)."""
    items = np.ascontiguousarray(items, dtype=np.uint64)
    values = np.ascontiguousarray(values, dtype=np.uint32)
    T = np.zeros((mu, 1 << logb), dtype=np.uint64)
    V = np.zeros((mu, 1 << logb), dtype=np.uint32)
    load = C.c_uint32(0)
    rc = lib().or_simple_hash_values(hash_key, lambda_bar, logb, items if len(items) else np.zeros(1, np.uint64),
                                     values if len(values) else np.zeros(1, np.uint32), len(items), mu, T, V,
                                     C.byref(load))
    return rc, T, V, int(load.value)


def mu_bound(n: int, b: int) -> int:
    """Server maximum bin load: the paper's value for its own (n, b) pairs,
    else smallest mu with b * P[Binomial(3n, 1/b) > mu] <= 2^-40."""
    if (n, b) in PAPER_MU:
        return PAPER_MU[(n, b)]
    from scipy.stats import binom as _binom
    trials, p = 3 * n, 1.0 / b
    mu = max(1, int(trials * p))
    while b * _binom.sf(mu, trials, p) > 2.0 ** -40:
        mu += 1
    return mu


class Ctx:
    """One BFV parameter set (N, t, prime bit sizes) plus PEPSI's code and
    hashing parameters."""

    def __init__(self, N, t, prime_bits, h=2, ell=0, lambda_bar=16, mu=0, hash_key=0, n_server=None, bins=0,
                 gamma=1):
        self.N, self.t, self.h = int(N), int(t), int(h)
        self.gamma = int(gamma)  # client maximum bin load (Table 2)
        self.prime_bits = list(prime_bits)
        self.k = len(self.prime_bits)
        self.lambda_bar = int(lambda_bar)
        self.ell = int(ell) if ell else code_length(lambda_bar, h)
        # b bins in B = b / N blocks of N slots (Section 4: ceil(b/N) ciphertexts per code bit)
        self.bins = int(bins) if bins else self.N
        self.blocks = self.bins // self.N
        self.logb = int(math.log2(self.bins))
        self.hash_key = int(hash_key)
        self.mu = int(mu) if mu else (mu_bound(n_server, self.bins) if n_server else 0)
        bits = np.array(self.prime_bits, dtype=np.uint8)
        self._p = lib().or_create(self.N, self.t, self.k, bits)
        if not self._p:
            raise ValueError("oracle: unsupported parameters")
        q = np.zeros(self.k, np.uint64)
        psi = np.zeros(self.k, np.uint64)
        tp = np.zeros(1, np.uint64)
        na = np.zeros(1, np.uint32)
        qa = np.zeros(32, np.uint64)
        lib().or_info(self._p, q, psi, tp, na, qa)
        self.q = [int(x) for x in q]
        self.psi = [int(x) for x in psi]
        self.psi_t = int(tp[0])
        self.aux = [int(x) for x in qa[: int(na[0])]]
        self.Q = math.prod(self.q)
        self.log2_q = lib().or_log2_q(self._p)
        if binom(self.ell, self.h) < (1 << self.lambda_bar):
            raise ValueError("C(ell,h) < 2^lambda_bar: CW-Encode would not be injective")

    def __del__(self):
        if getattr(self, "_p", None):
            lib().or_free(self._p)
            self._p = None

    # ---- shapes
    def ct_shape(self, comps=2):
        return (comps, self.k, self.N)

    # ---- encoding
    def encode(self, slots):
        s = np.ascontiguousarray(slots, dtype=np.uint32)
        m = np.zeros(self.N, np.uint32)
        lib().or_encode(self._p, s, m)
        return m

    def decode(self, m):
        m = np.ascontiguousarray(m, dtype=np.uint32)
        s = np.zeros(self.N, np.uint32)
        lib().or_decode(self._p, m, s)
        return s

    # ---- keys / encryption
    def keygen(self, seed):
        s = np.zeros(self.N, np.int8)
        rlk = np.zeros((self.k, 2, self.k, self.N), np.uint64)
        lib().or_keygen(self._p, seed, s, rlk)
        return s, rlk

    def encrypt(self, s, m, seed):
        """m: [count][N] plaintext coefficients in [0,t) -> [count][2][k][N]."""
        m = np.ascontiguousarray(np.atleast_2d(m), dtype=np.uint32)
        cts = np.zeros((m.shape[0], 2, self.k, self.N), np.uint64)
        lib().or_encrypt(self._p, np.ascontiguousarray(s, np.int8), m, m.shape[0], seed, cts)
        return cts

    def decrypt(self, s, ct):
        """Slots and noise budget of a ciphertext [2][r][N] over the first r
        primes (r = k, or fewer after modulus switching)."""
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        slots = np.zeros(self.N, np.uint32)
        b = C.c_double(0)
        rc = lib().or_decrypt_primes(self._p, np.ascontiguousarray(s, np.int8), ct, ct.shape[-2], slots, C.byref(b))
        assert rc == 0
        return slots, b.value

    def mod_switch(self, ct, r):
        """round(c~ * Q_r / Q) to the first r primes: [2][k][N] -> [2][r][N]."""
        out = np.zeros((2, r, self.N), np.uint64)
        rc = lib().or_mod_switch(self._p, np.ascontiguousarray(ct, np.uint64), r, out)
        assert rc == 0
        return out

    # ---- homomorphic primitives
    def pt_lift(self, m):
        out = np.zeros((self.k, self.N), np.uint64)
        lib().or_pt_lift(self._p, np.ascontiguousarray(m, np.uint32), out)
        return out

    def ct_mul_pt(self, ct, m):
        out = np.zeros((2, self.k, self.N), np.uint64)
        lib().or_ct_mul_pt(self._p, np.ascontiguousarray(ct, np.uint64), np.ascontiguousarray(m, np.uint32), out)
        return out

    def ct_axpy(self, a, z, b, ncomp=2):
        out = np.zeros_like(np.ascontiguousarray(a, np.uint64))
        lib().or_ct_axpy(self._p, np.ascontiguousarray(a, np.uint64), int(z), np.ascontiguousarray(b, np.uint64),
                         ncomp, out)
        return out

    def ct_add_const(self, ct, v):
        ct = np.array(ct, dtype=np.uint64)
        lib().or_ct_add_const(self._p, ct, int(v))
        return ct

    def ct_mult(self, a, b):
        out = np.zeros((3, self.k, self.N), np.uint64)
        rc = lib().or_ct_mult(self._p, np.ascontiguousarray(a, np.uint64), np.ascontiguousarray(b, np.uint64), out)
        assert rc == 0
        return out

    def ct_mult_sum(self, a, b, v=None):
        """round(t/Q * sum_i v_i (x) a_i (x) b_i) mod Q with one rounding;
        a, b: [n][2][k][N]; v: [n][N] plaintext coefficients in [0, t)
        (centred lift) or None."""
        a = np.ascontiguousarray(a, np.uint64)
        b = np.ascontiguousarray(b, np.uint64)
        vv = None if v is None else np.ascontiguousarray(v, np.uint32)
        out = np.zeros((3, self.k, self.N), np.uint64)
        rc = lib().or_ct_mult_sum(self._p, a, b, None if vv is None else vv.ctypes.data, a.shape[0], out)
        assert rc == 0
        return out

    def relin(self, rlk, ct3):
        out = np.zeros((2, self.k, self.N), np.uint64)
        lib().or_relin(self._p, np.ascontiguousarray(rlk, np.uint64), np.ascontiguousarray(ct3, np.uint64), out)
        return out

    # ---- PEPSI
    def cuckoo(self, items):
        return cuckoo(self.hash_key, self.lambda_bar, self.logb, items, self.gamma)

    def server_table(self, items, mu=None):
        return simple_hash(self.hash_key, self.lambda_bar, self.logb, items, mu or self.mu)

    def server_table_values(self, items, values, mu=None):
        """(rc, T [mu][N], V [mu][N] values of the stored items, max load)."""
        return simple_hash_values(self.hash_key, self.lambda_bar, self.logb, items, values, mu or self.mu)

    def server_plaintext(self, T, layer, j):
        out = np.zeros((self.k, self.N), np.uint64)
        lib().or_server_plaintext(self._p, np.ascontiguousarray(T, np.uint64), self.ell, self.h, layer, j, out)
        return out

    def query_plaintexts(self, table_val):
        m = np.zeros((self.ell, self.N), np.uint32)
        lib().or_query_plaintexts(self._p, np.ascontiguousarray(table_val, np.uint64), self.ell, self.h, m)
        return m

    def query(self, s, items, enc_seed):
        """Client side: cuckoo into the b bins of gamma slots -> for each
        block of N bins and each client batch i (slot i of every bin; Section
        4) the CW bit planes -> encode -> encrypt (ciphertext i of the request
        from stream index i, the request ordered [block][batch][bit]).
        Returns (rc, cts [ell][2][k][N], with a leading [gamma] when gamma > 1
        and [B] when there are B > 1 blocks, bin_of_item = bin*gamma + slot)."""
        rc, table, where = self.cuckoo(items)
        if rc:
            return rc, None, where
        g = self.gamma
        cols = table.reshape(self.bins, g)
        m = np.concatenate([self.query_plaintexts(np.ascontiguousarray(cols[b * self.N:(b + 1) * self.N, i]))
                            for b in range(self.blocks) for i in range(g)])
        cts = self.encrypt(s, m, enc_seed)
        shape = ((self.blocks,) if self.blocks > 1 else ()) + ((g,) if g > 1 else ()) + (self.ell, 2, self.k, self.N)
        return 0, cts.reshape(shape), where

    def eval(self, rlk, cts, T, mode=0, mask_seed=0, layer0=0, nlayers=None, debug=False, group=1, acc=False,
             V=None):
        """Alg 2 over layers [layer0, layer0+nlayers).  Returns the result
        ciphertext [2][k][N] and, with debug, per-layer h' and E words (E
        only when group <= 1); with acc, also the layer sum before
        relinearisation [3][k][N].  group > 1 rounds the last product of
        runs of `group` consecutive layers once (lazy rescaling).  Modes 2
        (labelled PSI) and 3 (PSI-Sum) need the value table V [mu][N]."""
        mu = T.shape[0]
        nl = mu - layer0 if nlayers is None else nlayers
        lazy = group > 1 and self.h > 1
        out = np.zeros((2, self.k, self.N), np.uint64)
        counts = np.zeros(2, np.uint64)
        dh = np.zeros((nl, 2, self.k, self.N), np.uint64) if debug else None
        de = np.zeros((nl, 3, self.k, self.N), np.uint64) if debug and not lazy else None
        da = np.zeros((3, self.k, self.N), np.uint64) if acc else None
        Vc = None if V is None else np.ascontiguousarray(V, np.uint32)  # kept alive across the call
        rc = lib().or_eval(self._p, np.ascontiguousarray(rlk, np.uint64), np.ascontiguousarray(cts, np.uint64),
                           self.ell, self.h, np.ascontiguousarray(T, np.uint64),
                           None if Vc is None else Vc.ctypes.data, mu, layer0, nl,
                           mode, mask_seed, group, out, dh.ctypes.data if debug else None,
                           de.ctypes.data if de is not None else None, da.ctypes.data if acc else None, counts)
        if rc:
            raise RuntimeError("oracle eval failed: %d" % rc)
        self.last_counts = (int(counts[0]), int(counts[1]))
        res = (out, dh, de) if debug else (out,)
        if acc:
            res = res + (da,)
        return res if len(res) > 1 else res[0]


def set_threads(n: int):
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return lib().or_get_threads()
