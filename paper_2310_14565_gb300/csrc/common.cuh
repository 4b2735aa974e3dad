// Shared device types and modular arithmetic for the PEPSI GB300 library.
//
// Modular reduction follows published methods, written from their
// definitions:
//  - Shoup's precomputed-quotient multiplication (NTL) for a fixed operand w:
//    w' = floor(w 2^64 / q); r = w x - umulhi(w', x) q lies in [0, 2q).
//  - Barrett reduction (Barrett 1986): of a product of two values below
//    2^bits(q) with the one-word constant floor(2^(bits+63) / q), and of a
//    64-bit value with floor(2^64 / q); a 128-bit value as hi (2^64 mod q)
//    (Shoup) plus lo (Barrett).
//  - Harvey's lazy butterflies (Harvey 2014) keep NTT values in [0, 4q).
// All primes are below 2^61, so 4q < 2^63 and every lazy sum fits in 64 bits.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;

#define PEPSI_MAXQ 8   // ciphertext primes q_i
#define PEPSI_MAXB 12  // auxiliary primes p_j of the exact multiplication base
#define PEPSI_MAXP (PEPSI_MAXQ + PEPSI_MAXB + 1)  // + the plaintext modulus t
#define PEPSI_DUMMY 0xFFFFFFFFFFFFFFFFull
#define PEPSI_CW_NONE 0xFFFFu

// One modulus q of n = bits(q) bits (n <= 61): N^-1 (Shoup); the split point
// s = ceil(n/2) of the split operand format (hi << 32 | lo with x = hi 2^s +
// lo) used by the multiply-accumulate; and the reduction constants
// mu = floor(2^(n+63)/q), m64 = floor(2^64/q), c64 = 2^64 mod q (Shoup).
struct DevPrime {
  u64 q, ninv, ninvs, split, nbits, mu, m64, c64, c64s;
};
__host__ __device__ __forceinline__ u64 to_split(u64 x, u64 s) { return ((x >> s) << 32) | (x & ((1ull << s) - 1)); }
__host__ __device__ __forceinline__ u64 from_split(u64 w, u64 s) { return ((w >> 32) << s) | (w & 0xFFFFFFFFull); }

// Constants of the exact RNS conversions (all residues reduced, Shoup
// companions where the value multiplies a varying operand).
struct RnsConst {
  // Garner over Q: cq[i][j] = q_j^-1 mod q_i (j < i)
  u64 cq[PEPSI_MAXQ][PEPSI_MAXQ], cqs[PEPSI_MAXQ][PEPSI_MAXQ];
  // radices of Q in B for Horner's rule: qb[j][l] = q_l mod p_j (Shoup)
  u64 qb[PEPSI_MAXB][PEPSI_MAXQ], qbs[PEPSI_MAXB][PEPSI_MAXQ];
  u64 qhalf_dig[PEPSI_MAXQ];  // mixed-radix digits of (Q-1)/2 over Q
  u64 qmodb[PEPSI_MAXB];      // Q mod p_j
  u64 qhalf_b[PEPSI_MAXB];    // (Q-1)/2 mod p_j
  u64 qinv_b[PEPSI_MAXB], qinv_bs[PEPSI_MAXB];  // Q^-1 mod p_j
  u64 qhalf_q[PEPSI_MAXQ];    // (Q-1)/2 mod q_i
  u64 t_q[PEPSI_MAXQ], t_qs[PEPSI_MAXQ];        // t mod q_i
  u64 t_b[PEPSI_MAXB], t_bs[PEPSI_MAXB];        // t mod p_j
  // Garner over B
  u64 cb[PEPSI_MAXB][PEPSI_MAXB], cbs[PEPSI_MAXB][PEPSI_MAXB];
  u64 bq[PEPSI_MAXQ][PEPSI_MAXB], bqs[PEPSI_MAXQ][PEPSI_MAXB];  // p_l mod q_i (Shoup)
  u64 bhalf_dig[PEPSI_MAXB];        // mixed-radix digits of (B-1)/2 over B
  u64 bmodq[PEPSI_MAXQ];            // B mod q_i
  // decryption and encoding
  u64 pq_t[PEPSI_MAXQ];     // prod_{m<l} q_m mod t
  double pq_d[PEPSI_MAXQ];  // prod_{m<l} q_m as a double
  u64 qinv_t;               // Q^-1 mod t
  u64 qhalf_t;              // (Q-1)/2 mod t
  u64 qdt_q[PEPSI_MAXQ], qdt_qs[PEPSI_MAXQ];  // floor(Q/t) mod q_i
  u64 qmt;                  // Q mod t
};

// Primes (Q then B) and conversion constants passed by value to the exact
// RNS kernels, so that they are read from the kernel parameter space.
struct RnsArgs {
  DevPrime pr[PEPSI_MAXQ + PEPSI_MAXB];
  RnsConst rc;
  int N, k, kb;
};

// Everything a kernel needs to know about one parameter set.
struct DevView {
  int N, logN, k, kb, tidx;  // tidx: index of t among the moduli (= k + kb)
  const DevPrime* pr;        // [k + kb + 1]
  const ulonglong2* twp;     // [np][N] (psi^brev(i), its Shoup companion)
  const ulonglong2* itwp;    // [np][N] (psi^-brev(i), its Shoup companion); entry 0: psi^-brev(1) N^-1
  const RnsConst* rc;
  const RnsArgs* host_args;  // host copy for by-value launches (not dereferenced on the device)
  int nt;                    // threads per block of the ciphertext transforms (0: the default for N)
};

// ---------------------------------------------------------------- arithmetic
__device__ __forceinline__ u64 shoup_lazy(u64 x, u64 w, u64 ws, u64 q) {
  u64 qh = __umul64hi(x, ws);
  return x * w - qh * q;  // in [0, 2q)
}
__device__ __forceinline__ u64 shoup(u64 x, u64 w, u64 ws, u64 q) {
  u64 r = shoup_lazy(x, w, ws, q);
  return r >= q ? r - q : r;
}
// x mod q for any 64-bit x: one-word Barrett, floor(x m64 / 2^64) is short
// of floor(x/q) by at most 1.
__device__ __forceinline__ u64 barrett64(u64 x, const DevPrime& p) {
  const u64 r = x - __umul64hi(x, p.m64) * p.q;  // [0, 2q)
  return r >= p.q ? r - p.q : r;
}
// (hi:lo) mod q for any 128-bit value: hi 2^64 = hi c64 (mod q) by Shoup
// and lo by one-word Barrett, each in [0, 2q), then their sum reduced.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const DevPrime& p) {
  const u64 a = shoup_lazy(hi, p.c64, p.c64s, p.q);
  const u64 b = lo - __umul64hi(lo, p.m64) * p.q;
  const u64 q2 = 2 * p.q;
  u64 r = a + b;  // [0, 4q)
  r = r >= q2 ? r - q2 : r;
  return r >= p.q ? r - p.q : r;
}
// a b mod q for a, b < 2^n (Barrett 1973, one constant): x = a b < 2^2n,
// x1 = floor(x / 2^(n-1)) < 2^(n+1), and floor(x1 mu / 2^64) is short of
// floor(x/q) by at most 2 (the dropped fractions are below 1/4 and 1).
__device__ __forceinline__ u64 mulmod(u64 a, u64 b, const DevPrime& p) {
  const u64 lo = a * b, hi = __umul64hi(a, b);
  const int n = (int)p.nbits;
  const u64 x1 = (hi << (65 - n)) | (lo >> (n - 1));
  u64 r = lo - __umul64hi(x1, p.mu) * p.q;  // [0, 3q)
  const u64 q2 = 2 * p.q;
  r = r >= q2 ? r - q2 : r;
  return r >= p.q ? r - p.q : r;
}
__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q) {
  u64 s = a + b;
  return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
// 128-bit accumulate acc += a*b
__device__ __forceinline__ void mac128(u64& lo, u64& hi, u64 a, u64 b) {
  asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;" : "+l"(lo), "+l"(hi) : "l"(a), "l"(b));
}
__device__ __forceinline__ u32 brev_bits(u32 x, int bits) { return bits ? (__brev(x) >> (32 - bits)) : 0; }

// ------------------------------------------------------------- SplitMix64
// Counter-based use of SplitMix64 (Steele, Lea, Flood 2014): the idx-th
// output of a generator whose state starts at mix64(seed ^ mix64(stream)).
#define PEPSI_GOLDEN 0x9E3779B97F4A7C15ull
__host__ __device__ __forceinline__ u64 mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ u64 stream_key(u64 seed, u64 stream) { return mix64(seed ^ mix64(stream)); }
__host__ __device__ __forceinline__ u64 draw_keyed(u64 key, u64 idx) { return mix64(key + (idx + 1) * PEPSI_GOLDEN); }
// uniform in [0, bound) by rejection, attempt a at index pos*256 + a
__host__ __device__ __forceinline__ u64 sample_uniform(u64 key, u64 pos, u64 bound) {
  u64 rem = (0 - bound) % bound;
  u64 r = 0;
  for (u64 a = 0; a < 256; a++) {
    r = draw_keyed(key, (pos << 8) | a);
    if (rem == 0 || r < (u64)(0 - rem)) return r % bound;
  }
  return r % bound;
}
// centred binomial, eta = 21
__host__ __device__ __forceinline__ int sample_cbd21(u64 key, u64 pos) {
  u64 r = draw_keyed(key, pos);
#ifdef __CUDA_ARCH__
  return __popcll(r & 0x1FFFFFull) - __popcll((r >> 21) & 0x1FFFFFull);
#else
  return __builtin_popcountll(r & 0x1FFFFFull) - __builtin_popcountll((r >> 21) & 0x1FFFFFull);
#endif
}
__host__ __device__ __forceinline__ u64 make_stream(u64 purpose, u64 index, u64 prime) {
  return (purpose << 56) | (index << 8) | prime;
}
enum { STREAM_SK = 1, STREAM_RLK_A = 2, STREAM_RLK_E = 3, STREAM_ENC_A = 4, STREAM_ENC_E = 5, STREAM_MASK = 6 };
