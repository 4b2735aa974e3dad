"""PEPSI server-side homomorphic evaluation (arXiv 2310.14565) on GB300.

Thin Python binding over the C ABI of ``include/pepsi.h``: every call
marshals arguments (numpy arrays for host buffers, torch CUDA tensors or raw
integers for device buffers) and forwards to ``libpepsi_gb300.so``.  All
computation runs in the library's CUDA kernels; there is no CPU fallback, and
calls fail loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpepsi_gb300.so")
_lib = None

OK, E_PARAM, E_BIN_OVERFLOW, E_CUCKOO_FAIL, E_NOMEM, E_CUDA, E_TIMEOUT, E_NOISE = range(8)
MODE_INDICATOR, MODE_CARDINALITY, MODE_LABELS, MODE_SUM = 0, 1, 2, 3
DUMMY = 0xFFFFFFFFFFFFFFFF


class PepsiError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        detail = ""
        if code in (E_CUDA, E_NOMEM):
            try:
                detail = " [%s]" % lib().pepsi_last_error().decode()
            except Exception:
                pass
        super().__init__("%s failed: %s (code %d)%s" % (what, strerror(code), code, detail))


class Params(C.Structure):
    _fields_ = [
        ("N", C.c_uint32), ("t", C.c_uint64), ("k", C.c_uint32), ("prime_bits", C.c_uint8 * 8),
        ("h", C.c_uint32), ("ell", C.c_uint32), ("lambda_bar", C.c_uint32), ("num_hashes", C.c_uint32),
        ("mu", C.c_uint32), ("hash_key", C.c_uint64), ("resident_bytes", C.c_uint64),
        ("rescale_group", C.c_uint32), ("server_values", C.c_uint32), ("response_primes", C.c_uint32),
        ("bins", C.c_uint32), ("plaintext_bytes", C.c_uint32), ("gamma", C.c_uint32),
        ("client_cuckoo", C.c_uint32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("N", C.c_uint32), ("k", C.c_uint32), ("kb", C.c_uint32), ("ell", C.c_uint32), ("h", C.c_uint32),
        ("mu", C.c_uint32), ("lambda_bar", C.c_uint32), ("logb", C.c_uint32), ("t", C.c_uint64),
        ("q", C.c_uint64 * 8), ("psi", C.c_uint64 * 8), ("psi_t", C.c_uint64), ("b_primes", C.c_uint64 * 12),
        ("log2_q", C.c_double), ("rescale_group", C.c_uint32), ("rescale_cap", C.c_uint32),
        ("response_primes", C.c_uint32), ("bins", C.c_uint32), ("blocks", C.c_uint32),
        ("plaintext_bytes", C.c_uint32), ("gamma", C.c_uint32),
    ]


class Schedule(C.Structure):
    _fields_ = [("chunk", C.c_uint32), ("ntt_threads", C.c_uint32), ("relin_fused", C.c_uint32),
                ("batch_points", C.c_uint32), ("batch_groups", C.c_uint32), ("batch_requests", C.c_uint32)]


class LaneDesc(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("set_id", C.c_int), ("slots", C.c_uint32)]


class EngineStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("steps", C.c_uint64),
                ("bytes_in_use", C.c_uint64), ("bytes_peak", C.c_uint64), ("budget", C.c_uint64)]


RESCALE_ALL = 0xFFFFFFFF

SYMBOLS = {
    # name: (restype, argtypes)
    "pepsi_setup": (C.c_int, [C.POINTER(Params), C.c_uint64, C.POINTER(C.c_void_p)]),
    "pepsi_get_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "pepsi_set_rescale_group": (C.c_int, [C.c_void_p, C.c_uint32]),
    "pepsi_get_schedule": (C.c_int, [C.c_void_p, C.POINTER(Schedule)]),
    "pepsi_set_schedule": (C.c_int, [C.c_void_p, C.POINTER(Schedule)]),
    "pepsi_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_uint32)]),
    "pepsi_wait_probe": (C.c_int, [C.c_void_p, C.c_int]),
    "pepsi_request_bits": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint64, C.POINTER(C.c_double),
                                     C.POINTER(C.c_uint64), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "pepsi_comm_optimal_h": (C.c_int, [C.c_uint32, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint32)]),
    "pepsi_server_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_int)]),
    "pepsi_server_table": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "pepsi_server_load_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_int)]),
    "pepsi_server_values": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "pepsi_server_plaintexts": (C.c_int, [C.c_void_p, C.c_int, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p]),
    "pepsi_query": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pepsi_eval": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_uint64, C.c_void_p, C.c_void_p]),
    "pepsi_eval_batch": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_int), C.POINTER(C.c_uint64), C.POINTER(C.c_void_p), C.c_void_p]),
    "pepsi_eval_layers": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "pepsi_decrypt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "pepsi_decrypt_primes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.POINTER(C.c_double)]),
    "pepsi_mod_switch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_uint32, C.c_void_p, C.c_void_p]),
    "pepsi_ntt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]),
    "pepsi_ct_mult": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p]),
    "pepsi_relin": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "pepsi_relin_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    "pepsi_export_keys": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pepsi_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "pepsi_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_char_p), C.POINTER(C.c_uint64),
                                     C.POINTER(C.c_double), C.c_int]),
    "pepsi_int_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "pepsi_engine_create": (C.c_int, [C.POINTER(LaneDesc), C.c_int, C.c_uint64, C.POINTER(C.c_void_p)]),
    "pepsi_engine_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_uint64, C.c_void_p,
                                      C.POINTER(C.c_uint64)]),
    "pepsi_engine_pump": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "pepsi_engine_run": (C.c_int, [C.c_void_p]),
    "pepsi_engine_start": (C.c_int, [C.c_void_p]),
    "pepsi_engine_stop": (C.c_int, [C.c_void_p]),
    "pepsi_engine_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_double)]),
    "pepsi_engine_get_stats": (C.c_int, [C.c_void_p, C.POINTER(EngineStats)]),
    "pepsi_engine_fail_next": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "pepsi_engine_destroy": (None, [C.c_void_p]),
    "pepsi_engine_capture": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pepsi_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "pepsi_graph_destroy": (None, [C.c_void_p]),
    "pepsi_destroy": (None, [C.c_void_p]),
    "pepsi_strerror": (C.c_char_p, [C.c_int]),
    "pepsi_last_error": (C.c_char_p, []),
}


def lib():
    """Load the CUDA library; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpepsi_gb300.so is missing: build it with paper_2310_14565_gb300.build.build() "
                               "(requires nvcc); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SYMBOLS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().pepsi_strerror(code).decode()
    except RuntimeError:
        return "error %d" % code


def _need(x, words, what):
    """Reject a numpy array or torch tensor smaller than `words` 64-bit words
    (the C ABI takes raw pointers and cannot check); raw integer pointers
    are the caller's responsibility."""
    if x is None or isinstance(x, int):
        return
    if isinstance(x, np.ndarray):
        n, item = x.size, x.itemsize
    elif hasattr(x, "numel"):
        n, item = int(x.numel()), int(x.element_size())
    else:
        return
    if item != 8 or n < words:
        raise ValueError("%s: need %d 64-bit words, got %d elements of %d bytes" % (what, words, n, item))


def _ptr(x):
    """Address of a numpy array, a torch tensor or an integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("unsupported buffer type %r" % type(x))


def _stream(s):
    """cudaStream_t for a call: an explicit stream, else torch's current
    stream when torch has initialised CUDA (so device tensors produced by
    torch are ordered before the call), else the context's own stream."""
    if s is None:
        torch = sys.modules.get("torch")
        if torch is not None and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream or None
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _check(rc, what):
    if rc != OK:
        raise PepsiError(rc, what)


def request_bits(lambda_bar, h, bins):
    """Request size model of Section 6.1: (bits, ell, log2 N, log2 q)."""
    b, l, ln, lq = C.c_double(0), C.c_uint64(0), C.c_uint32(0), C.c_uint32(0)
    _check(lib().pepsi_request_bits(lambda_bar, h, bins, C.byref(b), C.byref(l), C.byref(ln), C.byref(lq)),
           "pepsi_request_bits")
    return b.value, int(l.value), int(ln.value), int(lq.value)


def comm_optimal_h(lambda_bar, bins, h_max=64):
    """Hamming weight minimising the request size (ties to the smaller h)."""
    h = C.c_uint32(0)
    _check(lib().pepsi_comm_optimal_h(lambda_bar, bins, h_max, C.byref(h)), "pepsi_comm_optimal_h")
    return int(h.value)


INT_MAD_LO, INT_MAD_WIDE, INT_MUL_WIDE = 0, 1, 2


def int_peak(form=INT_MAD_WIDE):
    """Measured integer multiply throughput of the current GPU (ops/s):
    INT_MAD_WIDE (32x32->64 multiply-add into a 64-bit sum), INT_MUL_WIDE
    (the wide product alone) or INT_MAD_LO (32-bit multiply-add)."""
    v = C.c_double(0)
    _check(lib().pepsi_int_peak(int(form), C.byref(v)), "pepsi_int_peak")
    return v.value


class Context:
    """One parameter set with its keys, server sets and scratch (pepsi_ctx)."""

    def __init__(self, N, t=65537, prime_bits=(36, 36, 37), h=2, ell=0, lambda_bar=16, mu=0, hash_key=0,
                 key_seed=3, resident_bytes=0, rescale_group=0, server_values=0, response_primes=0, bins=0, plaintext_bytes=0,
                 gamma=0, client_cuckoo=0):
        p = Params()
        p.N, p.t, p.k = N, t, len(prime_bits)
        for i, b in enumerate(prime_bits):
            p.prime_bits[i] = b
        p.h, p.ell, p.lambda_bar, p.num_hashes, p.mu = h, ell, lambda_bar, 3, mu
        p.hash_key, p.resident_bytes, p.rescale_group = hash_key, resident_bytes, rescale_group
        p.server_values, p.response_primes, p.bins = server_values, response_primes, bins
        p.plaintext_bytes = plaintext_bytes
        p.gamma = gamma
        p.client_cuckoo = client_cuckoo
        self._h = C.c_void_p()
        _check(lib().pepsi_setup(C.byref(p), key_seed, C.byref(self._h)), "pepsi_setup")
        info = Info()
        _check(lib().pepsi_get_info(self._h, C.byref(info)), "pepsi_get_info")
        self.N, self.k, self.kb, self.ell, self.h = info.N, info.k, info.kb, info.ell, info.h
        self.t, self.log2_q = info.t, info.log2_q
        self.q = [int(info.q[i]) for i in range(self.k)]
        self.psi = [int(info.psi[i]) for i in range(self.k)]
        self.psi_t = int(info.psi_t)
        self.b_primes = [int(info.b_primes[i]) for i in range(min(self.kb, 12))]
        self.rescale_cap = int(info.rescale_cap)
        self.response_primes = int(info.response_primes)
        self.bins, self.blocks = int(info.bins), int(info.blocks)
        self.plaintext_bytes = int(info.plaintext_bytes)
        self.gamma = int(info.gamma)
        self.mu = {}

    def close(self):
        if self._h:
            lib().pepsi_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- shapes
    def ct_words(self, comps=2):
        return comps * self.k * self.N

    def wait_probe(self, arrive):
        """Status code of the bounded-wait test (OK, or E_TIMEOUT when
        nothing completes the barrier)."""
        return lib().pepsi_wait_probe(self._h, int(arrive))

    def set_rescale_group(self, group):
        """Rounding run length of later evaluations (1: per layer;
        RESCALE_ALL: one rounding per evaluation), cut at rescale_cap."""
        _check(lib().pepsi_set_rescale_group(self._h, int(group)), "pepsi_set_rescale_group")

    def schedule(self):
        """The evaluation schedule: {chunk, ntt_threads, relin_fused}."""
        sc = Schedule()
        _check(lib().pepsi_get_schedule(self._h, C.byref(sc)), "pepsi_get_schedule")
        return {"chunk": int(sc.chunk), "ntt_threads": int(sc.ntt_threads), "relin_fused": int(sc.relin_fused),
                "batch_points": int(sc.batch_points), "batch_groups": int(sc.batch_groups),
                "batch_requests": int(sc.batch_requests)}

    def set_schedule(self, chunk=None, ntt_threads=None, relin_fused=None, batch_points=None, batch_groups=None,
                     batch_requests=None):
        """Change fields of the evaluation schedule (None keeps a field);
        the result words never depend on it."""
        cur = self.schedule()
        sc = Schedule()
        sc.chunk = cur["chunk"] if chunk is None else int(chunk)
        sc.ntt_threads = cur["ntt_threads"] if ntt_threads is None else int(ntt_threads)
        sc.relin_fused = cur["relin_fused"] if relin_fused is None else int(relin_fused)
        sc.batch_points = cur["batch_points"] if batch_points is None else int(batch_points)
        sc.batch_groups = cur["batch_groups"] if batch_groups is None else int(batch_groups)
        sc.batch_requests = cur["batch_requests"] if batch_requests is None else int(batch_requests)
        _check(lib().pepsi_set_schedule(self._h, C.byref(sc)), "pepsi_set_schedule")

    # ---- server side
    def server_load(self, items):
        items = np.ascontiguousarray(items, dtype=np.uint64)
        sid = C.c_int(-1)
        _check(lib().pepsi_server_load(self._h, _ptr(items) if items.size else None, items.size, C.byref(sid)),
               "pepsi_server_load")
        return sid.value

    def server_load_values(self, items, values):
        """Server set with a value in [0, t) per item (labelled PSI / PSI-Sum)."""
        items = np.ascontiguousarray(items, dtype=np.uint64)
        values = np.ascontiguousarray(values, dtype=np.uint32)
        if values.shape != items.shape:
            raise ValueError("one value per item")
        sid = C.c_int(-1)
        _check(lib().pepsi_server_load_values(self._h, _ptr(items) if items.size else None,
                                              _ptr(values) if values.size else None, items.size, C.byref(sid)),
               "pepsi_server_load_values")
        return sid.value

    def _blocked(self, shape):
        """Array shape with a leading block dimension when b > N."""
        return (self.blocks,) + tuple(shape) if self.blocks > 1 else tuple(shape)

    def _batched(self, shape):
        """Request / response shape: [B] when b > N, then [gamma] when the
        client bins hold gamma > 1 items (one ciphertext set per batch)."""
        lead = ((self.blocks,) if self.blocks > 1 else ()) + ((self.gamma,) if self.gamma > 1 else ())
        return lead + tuple(shape)

    def server_values(self, set_id, mu):
        out = np.zeros((mu, self.bins), dtype=np.uint32)
        _check(lib().pepsi_server_values(self._h, set_id, _ptr(out)), "pepsi_server_values")
        return out

    def server_table(self, set_id, mu):
        out = np.zeros((mu, self.bins), dtype=np.uint64)
        _check(lib().pepsi_server_table(self._h, set_id, _ptr(out)), "pepsi_server_table")
        return out

    def server_plaintexts(self, set_id, layer0, nl, out=None, stream=None):
        if out is None:
            out = np.zeros(self._blocked((nl, self.ell, self.k, self.N)), dtype=np.uint64)
        _need(out, self.blocks * nl * self.ell * self.k * self.N, "server_plaintexts out")
        _check(lib().pepsi_server_plaintexts(self._h, set_id, layer0, nl, _ptr(out), _stream(stream)),
               "pepsi_server_plaintexts")
        return out

    # ---- client side
    def query(self, items, enc_seed, out=None, stream=None):
        items = np.ascontiguousarray(items, dtype=np.uint64)
        if out is None:
            out = np.zeros(self._batched((self.ell, 2, self.k, self.N)), dtype=np.uint64)
        _need(out, self._request_words(), "query out")
        where = np.full(max(items.size, 1), -1, dtype=np.int32)
        _check(lib().pepsi_query(self._h, _ptr(items) if items.size else None, items.size, enc_seed, _ptr(out),
                                 _ptr(where), _stream(stream)), "pepsi_query")
        return out, where[: items.size]

    def decrypt(self, ct):
        """Slots and noise budget of a ciphertext [2][r][N] over the first r
        primes (r = k, or fewer for a switched response).  A response of B
        blocks [B][2][r][N] gives the B*N slots in bin order and the
        smallest budget; one of gamma > 1 client batches ([gamma][2][r][N],
        or [B][gamma][2][r][N]) gives bins * gamma slots in the order of
        query's bin_of_item, bin * gamma + batch."""
        if self.gamma > 1 and len(ct.shape) == (5 if self.blocks > 1 else 4):
            nb = self.blocks
            cts = ct.reshape((nb, self.gamma) + tuple(ct.shape[-3:]))
            parts = [[self.decrypt(cts[b, i]) for i in range(self.gamma)] for b in range(nb)]
            slots = np.stack([np.stack([p[0] for p in row], axis=1) for row in parts]).reshape(-1)
            return slots, min(p[1] for row in parts for p in row)
        if len(ct.shape) == 4:
            parts = [self.decrypt(ct[i]) for i in range(int(ct.shape[0]))]
            return np.concatenate([p[0] for p in parts]), min(p[1] for p in parts)
        ct = np.ascontiguousarray(ct, dtype=np.uint64) if isinstance(ct, np.ndarray) else ct
        r = int(ct.shape[-2])
        if int(ct.shape[-1]) != self.N or not 1 <= r <= self.k:
            raise ValueError("decrypt: a ciphertext is [2][r][N] with 1 <= r <= k")
        _need(ct, 2 * r * self.N, "decrypt ct")
        slots = np.zeros(self.N, dtype=np.uint32)
        b = C.c_double(0)
        rc = lib().pepsi_decrypt_primes(self._h, _ptr(ct), r, _ptr(slots), C.byref(b))
        if rc not in (OK, E_NOISE):
            raise PepsiError(rc, "pepsi_decrypt_primes")
        return slots, b.value

    def mod_switch(self, cts, r, out=None, stream=None):
        """round(c~ Q_r / Q): [n][2][k][N] (or [2][k][N]) -> [n][2][r][N]."""
        single = len(cts.shape) == 3
        n = 1 if single else int(cts.shape[0])
        if out is None:
            out = np.zeros(((2, r, self.N) if single else (n, 2, r, self.N)), dtype=np.uint64)
            if isinstance(cts, np.ndarray):
                cts = np.ascontiguousarray(cts, dtype=np.uint64)
        _need(cts, n * 2 * self.k * self.N, "mod_switch cts")
        _need(out, n * 2 * r * self.N, "mod_switch out")
        _check(lib().pepsi_mod_switch(self._h, _ptr(cts), n, r, _ptr(out), _stream(stream)), "pepsi_mod_switch")
        return out

    # ---- evaluation
    def _request_words(self):
        return self.blocks * self.gamma * self.ell * 2 * self.k * self.N

    def _response_words(self):
        return self.blocks * self.gamma * 2 * self.response_primes * self.N

    def eval(self, set_id, cts, mode=MODE_INDICATOR, mask_seed=0, out=None, stream=None):
        if out is None:
            out = np.zeros(self._batched((2, self.response_primes, self.N)), dtype=np.uint64)
        _need(cts, self._request_words(), "eval cts")
        _need(out, self._response_words(), "eval out")
        _check(lib().pepsi_eval(self._h, set_id, _ptr(cts), mode, mask_seed, _ptr(out), _stream(stream)),
               "pepsi_eval")
        return out

    def autotune(self, set_id, cts, stream=None):
        """Time the evaluation at layer chunks of 32..256, keep the fastest;
        returns the chosen chunk (outputs do not depend on it)."""
        _need(cts, self._request_words(), "autotune cts")
        chosen = C.c_uint32(0)
        _check(lib().pepsi_autotune(self._h, set_id, _ptr(cts), _stream(stream), C.byref(chosen)), "pepsi_autotune")
        return int(chosen.value)

    def eval_batch(self, set_ids, cts_list, modes=None, mask_seeds=None, outs=None, stream=None):
        """pepsi_eval_batch: one output ciphertext per request."""
        nq = len(cts_list)
        if outs is None:
            outs = [np.zeros(self._batched((2, self.response_primes, self.N)), dtype=np.uint64) for _ in range(nq)]
        for x, o in zip(cts_list, outs):
            _need(x, self._request_words(), "eval_batch cts")
            _need(o, self._response_words(), "eval_batch out")
        sid = (C.c_int * nq)(*set_ids)
        cp = (C.c_void_p * nq)(*[_ptr(x) for x in cts_list])
        op = (C.c_void_p * nq)(*[_ptr(x) for x in outs])
        md = (C.c_int * nq)(*modes) if modes is not None else None
        ms = (C.c_uint64 * nq)(*mask_seeds) if mask_seeds is not None else None
        _check(lib().pepsi_eval_batch(self._h, nq, sid, cp, md, ms, op, _stream(stream)), "pepsi_eval_batch")
        return outs

    def eval_layers(self, set_id, cts, layer0, nl, want_h=True, want_e=True, stream=None):
        h = np.zeros(self._batched((nl, 2, self.k, self.N)), dtype=np.uint64) if want_h else None
        e = np.zeros(self._batched((nl, 3, self.k, self.N)), dtype=np.uint64) if want_e else None
        _need(cts, self._request_words(), "eval_layers cts")
        _check(lib().pepsi_eval_layers(self._h, set_id, _ptr(cts), layer0, nl, _ptr(h), _ptr(e), _stream(stream)),
               "pepsi_eval_layers")
        return h, e

    # ---- primitives (device buffers)
    def ntt(self, polys, count, inverse=False, stream=None):
        _need(polys, count * self.k * self.N, "ntt polys")
        _check(lib().pepsi_ntt(self._h, _ptr(polys), count, int(inverse), _stream(stream)), "pepsi_ntt")

    def ct_mult(self, a, b, n, out, relin=False, stream=None):
        ct2 = 2 * self.k * self.N
        _need(a, n * ct2, "ct_mult a")
        _need(b, n * ct2, "ct_mult b")
        _need(out, n * (2 if relin else 3) * self.k * self.N, "ct_mult out")
        _check(lib().pepsi_ct_mult(self._h, _ptr(a), _ptr(b), n, int(relin), _ptr(out), _stream(stream)),
               "pepsi_ct_mult")

    def relin(self, ct3, n, out, stream=None):
        _need(ct3, n * 3 * self.k * self.N, "relin input")
        _need(out, n * 2 * self.k * self.N, "relin out")
        _check(lib().pepsi_relin(self._h, _ptr(ct3), n, _ptr(out), _stream(stream)), "pepsi_relin")

    def relin_noalloc(self, ct3, n, out, stream=None):
        """pepsi_relin without any allocation: scratch in the library's fixed
        16 MiB device array (shared by all calls; do not overlap calls)."""
        _need(ct3, n * 3 * self.k * self.N, "relin_noalloc input")
        _need(out, n * 2 * self.k * self.N, "relin_noalloc out")
        rc = lib().pepsi_relin_noalloc(self._h, _ptr(ct3), n, _ptr(out), _stream(stream))
        if rc != OK:
            err = PepsiError(rc, "pepsi_relin_noalloc")
            if rc == E_PARAM:
                err.args = (err.args[0] + " [%s]" % lib().pepsi_last_error().decode(),)
            raise err

    def export_keys(self):
        s = np.zeros(self.N, dtype=np.int8)
        rlk = np.zeros((self.k, 2, self.k, self.N), dtype=np.uint64)
        _check(lib().pepsi_export_keys(self._h, _ptr(s), _ptr(rlk)), "pepsi_export_keys")
        return s, rlk

    # ---- profiling
    def profile(self, on=True):
        _check(lib().pepsi_profile_enable(self._h, int(on)), "pepsi_profile_enable")

    def profile_read(self):
        n = 16
        names = (C.c_char_p * n)()
        launches = (C.c_uint64 * n)()
        ms = (C.c_double * n)()
        cnt = lib().pepsi_profile_read(self._h, names, launches, ms, n)
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(cnt)}


class Engine:
    """Continuous-batching request engine (pepsi_engine_*): lanes of
    (Context, set id, slots); every request's result has the words of
    Context.eval.  Keeps the contexts and the buffers of requests in flight
    alive until they are waited for."""

    def __init__(self, lanes, hbm_budget=0):
        self._ctxs = [lc for lc, _, _ in lanes]
        arr = (LaneDesc * len(lanes))()
        for i, (ctx, sid, slots) in enumerate(lanes):
            arr[i].ctx, arr[i].set_id, arr[i].slots = ctx._h.value, sid, slots
        self._h = C.c_void_p()
        _check(lib().pepsi_engine_create(arr, len(lanes), hbm_budget, C.byref(self._h)), "pepsi_engine_create")
        self._lane_ctx = [ctx for ctx, _, _ in lanes]
        self._held = {}

    def submit(self, lane, cts, out=None, mode=MODE_INDICATOR, mask_seed=0):
        """Queue a request; returns (ticket, out).  cts [ell][2][k][N] and
        out [2][r][N]: numpy (pinned is best) or torch CUDA tensors."""
        ctx = self._lane_ctx[lane]
        if out is None:
            out = np.zeros((2, ctx.response_primes, ctx.N), dtype=np.uint64)
        _need(cts, ctx.ell * 2 * ctx.k * ctx.N, "engine cts")
        _need(out, 2 * ctx.response_primes * ctx.N, "engine out")
        t = C.c_uint64(0)
        _check(lib().pepsi_engine_submit(self._h, lane, _ptr(cts), mode, mask_seed, _ptr(out), C.byref(t)),
               "pepsi_engine_submit")
        self._held[t.value] = (cts, out)
        return t.value, out

    def pump(self):
        """One scheduling pass; returns the number of requests not yet done."""
        p = C.c_uint64(0)
        _check(lib().pepsi_engine_pump(self._h, C.byref(p)), "pepsi_engine_pump")
        return int(p.value)

    def run(self):
        _check(lib().pepsi_engine_run(self._h), "pepsi_engine_run")

    def start(self):
        _check(lib().pepsi_engine_start(self._h), "pepsi_engine_start")

    def stop(self):
        _check(lib().pepsi_engine_stop(self._h), "pepsi_engine_stop")

    def wait(self, ticket):
        """Block until the request is done; its latency in ms (submission to
        completion seen by the engine)."""
        ms = C.c_double(0)
        rc = lib().pepsi_engine_wait(self._h, ticket, C.byref(ms))
        self._held.pop(ticket, None)
        _check(rc, "pepsi_engine_wait")
        return ms.value

    def capture(self, stream=None):
        """Capture every submitted, not yet admitted request into one CUDA
        graph (device buffers only); returns an EngineGraph.  The requests'
        tickets are done; their outputs are written by each launch."""
        g = C.c_void_p()
        _check(lib().pepsi_engine_capture(self._h, _stream(stream), C.byref(g)), "pepsi_engine_capture")
        held = list(self._held.values())
        self._held.clear()
        return EngineGraph(g, self, held)

    def fail_next(self, lane, status):
        """Test hook: the lane's next admission fails on the host with status."""
        _check(lib().pepsi_engine_fail_next(self._h, lane, status), "pepsi_engine_fail_next")

    def stats(self):
        st = EngineStats()
        _check(lib().pepsi_engine_get_stats(self._h, C.byref(st)), "pepsi_engine_get_stats")
        return {f: int(getattr(st, f)) for f, _ in EngineStats._fields_}

    def close(self):
        if self._h:
            lib().pepsi_engine_destroy(self._h)
            self._h = C.c_void_p()
        self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class EngineGraph:
    """A captured engine schedule: launch() replays it on its buffers."""

    def __init__(self, handle, engine, held):
        self._h, self._engine, self._held = handle, engine, held

    def launch(self, stream=None, synchronize=True):
        _check(lib().pepsi_graph_launch(self._h, _stream(stream), int(synchronize)), "pepsi_graph_launch")

    def close(self):
        if self._h:
            lib().pepsi_graph_destroy(self._h)
            self._h = C.c_void_p()
        self._held = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
