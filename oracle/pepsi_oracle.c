/*
 * pepsi_oracle.c -- plain, slow CPU reference of PEPSI's server-side
 * evaluation (arXiv 2310.14565) in RNS-BFV.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Every function states the passage it follows.  Where the paper is silent
 * (prime choice, roots, hashing functions, randomness, CW mapping, slot
 * order) the function follows the reading written in its comment.
 *
 * Arithmetic is the textbook one: a*b mod q through a 128-bit product and
 * the `%` operator, big integers through schoolbook limbs and bit-serial
 * long division, CRT through Garner's mixed-radix method.  Ring products
 * mod a prime use a radix-2 NTT (a library-style primitive), checked in the
 * tests against the O(N^2) evaluation definition and against schoolbook
 * negacyclic convolution.
 *
 * Parity status: every function is pinned by a CPU test except the
 * ciphertext words of Mult/relin, which the paper does not fix (SEAL's own
 * rounding is not printed); those are pinned by decryption identities, the
 * noise bound and a brute-force big-integer recomputation at tiny N.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

#define OR_MAXK 16   /* ciphertext primes */
#define OR_MAXA 24   /* auxiliary primes for exact integer products */
#define BNL 48       /* 32-bit limbs per big integer: 1536 bits */
#define OR_DUMMY UINT64_MAX
#define OR_MAX_GROUP 65536 /* most layers whose rounding may be deferred to one */

enum { OR_OK = 0, OR_E_PARAM = 1, OR_E_BIN_OVERFLOW = 2, OR_E_CUCKOO_FAIL = 3, OR_E_NOMEM = 4 };

/* ------------------------------------------------------------------ */
/* modular arithmetic on u64 (textbook: 128-bit product, then %)        */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
/* addmod/submod take operands already reduced into [0, m) */
static u64 addmod(u64 a, u64 b, u64 m) { u64 s = a + b; return s >= m ? s - m : s; }
static u64 submod(u64 a, u64 b, u64 m) { return a >= b ? a - b : a + (m - b); }
static u64 powmod(u64 b, u64 e, u64 m) {
  u64 r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = mulmod(r, b, m);
    b = mulmod(b, b, m);
    e >>= 1;
  }
  return r;
}
/* inverse mod a prime by Fermat's little theorem */
static u64 invmod(u64 a, u64 p) { return powmod(a % p, p - 2, p); }
/* signed small integer to its residue in [0, m) */
static u64 smod(i64 v, u64 m) {
  if (v >= 0) return (u64)v % m;
  u64 r = ((u64)(-(v + 1)) + 1) % m;
  return r ? m - r : 0;
}

/* Miller-Rabin with the first twelve prime bases: deterministic below 2^64. */
int or_is_prime(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (n == bases[i]) return 1;
    if (n % bases[i] == 0) return 0;
  }
  u64 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; s++; }
  for (int i = 0; i < 12; i++) {
    u64 x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int comp = 1;
    for (int r = 1; r < s; r++) {
      x = mulmod(x, x, n);
      if (x == n - 1) { comp = 0; break; }
    }
    if (comp) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based stream  */
/* ------------------------------------------------------------------ */
#define GOLDEN 0x9E3779B97F4A7C15ULL
u64 or_mix64(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
/* idx-th output (0-based) of a SplitMix64 generator whose state starts at
 * mix64(seed XOR mix64(stream)). */
u64 or_draw(u64 seed, u64 stream, u64 idx) {
  u64 st = or_mix64(seed ^ or_mix64(stream));
  return or_mix64(st + (idx + 1) * GOLDEN);
}
/* Uniform value in [0, bound) for position pos: attempt a uses draw index
 * pos*256 + a and is accepted when it falls below the largest multiple of
 * bound that fits in 2^64 (rejection sampling). */
u64 or_sample_mod(u64 seed, u64 stream, u64 pos, u64 bound) {
  u64 rem = (0 - bound) % bound; /* 2^64 mod bound */
  u64 r = 0;
  for (u64 a = 0; a < 256; a++) {
    r = or_draw(seed, stream, (pos << 8) | a);
    if (rem == 0 || r < (u64)(0 - rem)) return r % bound;
  }
  return r % bound;
}
/* Centered binomial with eta = 21: popcount of 21 bits minus popcount of
 * the next 21 bits of one draw. */
int or_sample_cbd(u64 seed, u64 stream, u64 pos) {
  u64 r = or_draw(seed, stream, pos);
  return __builtin_popcountll(r & 0x1FFFFFULL) - __builtin_popcountll((r >> 21) & 0x1FFFFFULL);
}
/* Stream identifiers: purpose in the top byte, an index, a prime index. */
u64 or_stream(u64 purpose, u64 index, u64 prime) { return (purpose << 56) | (index << 8) | prime; }
enum { ST_SK = 1, ST_RLK_A = 2, ST_RLK_E = 3, ST_ENC_A = 4, ST_ENC_E = 5, ST_MASK = 6 };

/* ------------------------------------------------------------------ */
/* primes and roots                                                     */
/* ------------------------------------------------------------------ */
/* Largest prime q < 2^bits with q = 1 (mod 2N) that is not in `taken`. */
u64 or_find_prime(u32 bits, u32 N, const u64* taken, u32 ntaken) {
  u64 two_n = 2ULL * N;
  if (bits > 62 || (1ULL << bits) <= two_n) return 0;
  u64 q = (1ULL << bits) - two_n + 1;
  for (; q > two_n; q -= two_n) {
    int used = 0;
    for (u32 i = 0; i < ntaken; i++) used |= (taken[i] == q);
    if (!used && or_is_prime(q)) return q;
  }
  return 0;
}
/* Smallest w in [1, q) with w^N = -1 (mod q): the minimal primitive 2N-th
 * root of unity.  Any root w0 is found first; all others are w0^(2j+1). */
u64 or_min_root(u64 q, u32 N) {
  u64 e = (q - 1) / (2ULL * N);
  u64 w0 = 0;
  for (u64 g = 2; g < q; g++) {
    u64 w = powmod(g, e, q);
    if (powmod(w, N, q) == q - 1) { w0 = w; break; }
  }
  if (!w0) return 0;
  u64 w2 = mulmod(w0, w0, q), x = w0, best = w0;
  for (u32 j = 0; j < N; j++) {
    if (x < best) best = x;
    x = mulmod(x, w2, q);
  }
  return best;
}

static u32 brev(u32 x, u32 bits) {
  u32 r = 0;
  for (u32 i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}
static u32 ilog2(u32 n) { u32 l = 0; while ((1u << l) < n) l++; return l; }

/* ------------------------------------------------------------------ */
/* NTT over Z_q[X]/(X^N+1)                                             */
/* Definition: NTT(a)[i] = a(psi^(2*brev(i)+1)) mod q, i in [0, N).      */
/* ------------------------------------------------------------------ */
/* O(N^2) evaluation straight from the definition. */
void or_ntt_direct(const u64* a, u32 N, u64 q, u64 psi, u64* out) {
  u32 lg = ilog2(N);
  for (u32 i = 0; i < N; i++) {
    u64 x = powmod(psi, 2ULL * brev(i, lg) + 1, q), xp = 1, s = 0;
    for (u32 n = 0; n < N; n++) {
      s = addmod(s, mulmod(a[n] % q, xp, q), q);
      xp = mulmod(xp, x, q);
    }
    out[i] = s;
  }
}
typedef struct {
  u64 q, psi, ninv;
  u64* rev;  /* psi^brev(i) */
  u64* irev; /* psi^-brev(i) */
} ntt_tab;
static int tab_init(ntt_tab* T, u64 q, u32 N, u64 psi) {
  u32 lg = ilog2(N);
  T->q = q; T->psi = psi; T->ninv = invmod(N, q);
  T->rev = (u64*)malloc(sizeof(u64) * N);
  T->irev = (u64*)malloc(sizeof(u64) * N);
  if (!T->rev || !T->irev) return -1;
  u64 ipsi = invmod(psi, q);
  for (u32 i = 0; i < N; i++) {
    T->rev[i] = powmod(psi, brev(i, lg), q);
    T->irev[i] = powmod(ipsi, brev(i, lg), q);
  }
  return 0;
}
static void tab_free(ntt_tab* T) { free(T->rev); free(T->irev); T->rev = T->irev = NULL; }
/* Radix-2 Cooley-Tukey, natural order in, definition order out. */
static void ntt_fwd(u64* a, u32 N, const ntt_tab* T) {
  u64 q = T->q;
  for (u32 m = 1, len = N / 2; m < N; m <<= 1, len >>= 1)
    for (u32 i = 0; i < m; i++) {
      u64 w = T->rev[m + i];
      for (u32 j = 2 * i * len; j < 2 * i * len + len; j++) {
        u64 u = a[j], v = mulmod(a[j + len], w, q);
        a[j] = addmod(u, v, q);
        a[j + len] = submod(u, v, q);
      }
    }
}
/* Gentleman-Sande inverse of ntt_fwd, including the factor 1/N. */
static void ntt_inv(u64* a, u32 N, const ntt_tab* T) {
  u64 q = T->q;
  for (u32 m = N / 2, len = 1; m >= 1; m >>= 1, len <<= 1)
    for (u32 i = 0; i < m; i++) {
      u64 w = T->irev[m + i];
      for (u32 j = 2 * i * len; j < 2 * i * len + len; j++) {
        u64 u = a[j], v = a[j + len];
        a[j] = addmod(u, v, q);
        a[j + len] = mulmod(submod(u, v, q), w, q);
      }
    }
  for (u32 j = 0; j < N; j++) a[j] = mulmod(a[j], T->ninv, q);
}
/* Exported single-prime transforms for the tests (tables built per call). */
int or_ntt_fwd(u64* a, u32 N, u64 q, u64 psi) {
  ntt_tab T;
  if (tab_init(&T, q, N, psi)) return OR_E_NOMEM;
  ntt_fwd(a, N, &T);
  tab_free(&T);
  return 0;
}
int or_ntt_inv(u64* a, u32 N, u64 q, u64 psi) {
  ntt_tab T;
  if (tab_init(&T, q, N, psi)) return OR_E_NOMEM;
  ntt_inv(a, N, &T);
  tab_free(&T);
  return 0;
}
/* Negacyclic product c = a*b in Z_q[X]/(X^N+1) through the NTT. */
static void ring_mul(const u64* a, const u64* b, u64* c, u32 N, const ntt_tab* T, u64* tmp) {
  memcpy(c, a, sizeof(u64) * N);
  memcpy(tmp, b, sizeof(u64) * N);
  ntt_fwd(c, N, T);
  ntt_fwd(tmp, N, T);
  for (u32 i = 0; i < N; i++) c[i] = mulmod(c[i], tmp[i], T->q);
  ntt_inv(c, N, T);
}

/* ------------------------------------------------------------------ */
/* big integers: magnitude in 32-bit limbs, little-endian               */
/* ------------------------------------------------------------------ */
typedef struct { u32 d[BNL]; int n; } bn;          /* n = used limbs */
typedef struct { bn m; int neg; } sbn;             /* sign-magnitude */

static void bn_norm(bn* a) { while (a->n > 0 && a->d[a->n - 1] == 0) a->n--; }
static void bn_zero(bn* a) { memset(a, 0, sizeof(*a)); }
static void bn_set_u64(bn* a, u64 v) { bn_zero(a); a->d[0] = (u32)v; a->d[1] = (u32)(v >> 32); a->n = 2; bn_norm(a); }
static int bn_cmp(const bn* a, const bn* b) {
  if (a->n != b->n) return a->n > b->n ? 1 : -1;
  for (int i = a->n - 1; i >= 0; i--)
    if (a->d[i] != b->d[i]) return a->d[i] > b->d[i] ? 1 : -1;
  return 0;
}
static void bn_add(bn* r, const bn* a, const bn* b) {
  int n = a->n > b->n ? a->n : b->n;
  u64 c = 0;
  bn t;
  bn_zero(&t);
  for (int i = 0; i < n; i++) {
    c += (u64)(i < a->n ? a->d[i] : 0) + (i < b->n ? b->d[i] : 0);
    t.d[i] = (u32)c;
    c >>= 32;
  }
  t.n = n;
  if (c) t.d[t.n++] = (u32)c;
  *r = t;
}
/* r = a - b, requires a >= b */
static void bn_sub(bn* r, const bn* a, const bn* b) {
  i64 br = 0;
  bn t;
  bn_zero(&t);
  for (int i = 0; i < a->n; i++) {
    i64 v = (i64)a->d[i] - (i < b->n ? b->d[i] : 0) - br;
    br = v < 0;
    t.d[i] = (u32)(v + (br ? (1LL << 32) : 0));
  }
  t.n = a->n;
  bn_norm(&t);
  *r = t;
}
static void bn_mul_u64(bn* r, const bn* a, u64 m) {
  bn t;
  bn_zero(&t);
  u128 c = 0;
  int i;
  for (i = 0; i < a->n; i++) {
    c += (u128)a->d[i] * m;
    t.d[i] = (u32)c;
    c >>= 32;
  }
  while (c) { t.d[i++] = (u32)c; c >>= 32; }
  t.n = i;
  bn_norm(&t);
  *r = t;
}
static void bn_add_u64(bn* r, const bn* a, u64 v) { bn b; bn_set_u64(&b, v); bn_add(r, a, &b); }
static u64 bn_mod_u64(const bn* a, u64 q) {
  u128 r = 0;
  for (int i = a->n - 1; i >= 0; i--) r = ((r << 32) | a->d[i]) % q;
  return (u64)r;
}
static int bn_bitlen(const bn* a) {
  if (a->n == 0) return 0;
  return 32 * (a->n - 1) + (32 - __builtin_clz(a->d[a->n - 1]));
}
static int bn_bit(const bn* a, int i) { return (a->d[i >> 5] >> (i & 31)) & 1; }
static void bn_shl1_or(bn* a, int bit) {
  u32 c = (u32)bit;
  for (int i = 0; i < a->n; i++) {
    u32 nc = a->d[i] >> 31;
    a->d[i] = (a->d[i] << 1) | c;
    c = nc;
  }
  if (c) a->d[a->n++] = c;
}
/* Bit-serial long division: quo = floor(a / b), rem = a mod b (b > 0). */
static void bn_divmod(bn* quo, bn* rem, const bn* a, const bn* b) {
  bn q, r;
  bn_zero(&q);
  bn_zero(&r);
  int L = bn_bitlen(a);
  q.n = (L + 31) / 32;
  for (int i = L - 1; i >= 0; i--) {
    bn_shl1_or(&r, bn_bit(a, i));
    if (bn_cmp(&r, b) >= 0) {
      bn_sub(&r, &r, b);
      q.d[i >> 5] |= 1u << (i & 31);
    }
  }
  bn_norm(&q);
  if (quo) *quo = q;
  if (rem) *rem = r;
}
/* Short division by a word: quo = floor(a / d), returns a mod d. */
static u64 bn_div_u64(bn* quo, const bn* a, u64 d) {
  bn q;
  bn_zero(&q);
  u128 r = 0;
  for (int i = a->n - 1; i >= 0; i--) {
    r = (r << 32) | a->d[i];
    q.d[i] = (u32)(r / d);
    r %= d;
  }
  q.n = a->n;
  bn_norm(&q);
  if (quo) *quo = q;
  return (u64)r;
}
static double bn_log2(const bn* a) {
  if (a->n == 0) return -INFINITY;
  long double v = 0;
  int top = a->n - 1, lo = top - 3 < 0 ? 0 : top - 3;
  for (int i = top; i >= lo; i--) v = v * 4294967296.0L + a->d[i];
  return (double)(log2l(v) + 32.0L * lo);
}
/* signed helpers */
static void sbn_add(sbn* r, const sbn* a, const sbn* b) {
  if (a->neg == b->neg) { bn_add(&r->m, &a->m, &b->m); r->neg = a->neg; return; }
  int c = bn_cmp(&a->m, &b->m);
  if (c >= 0) { bn_sub(&r->m, &a->m, &b->m); r->neg = a->neg; }
  else { bn_sub(&r->m, &b->m, &a->m); r->neg = b->neg; }
  if (r->m.n == 0) r->neg = 0;
}
static u64 sbn_mod_u64(const sbn* a, u64 q) {
  u64 r = bn_mod_u64(&a->m, q);
  return (a->neg && r) ? q - r : r;
}

/* Garner's mixed-radix CRT: residues x[i] mod p[i] -> X in [0, prod p). */
static void crt_garner(const u64* x, const u64* p, u32 k, const u64* inv /* inv[i*k+j] = p_j^-1 mod p_i */, bn* X) {
  u64 v[OR_MAXA];
  for (u32 i = 0; i < k; i++) {
    u64 t = x[i] % p[i];
    for (u32 j = 0; j < i; j++) t = mulmod(submod(t, v[j] % p[i], p[i]), inv[i * k + j], p[i]);
    v[i] = t;
  }
  bn_set_u64(X, v[k - 1]);
  for (int i = (int)k - 2; i >= 0; i--) {
    bn_mul_u64(X, X, p[i]);
    bn_add_u64(X, X, v[i]);
  }
}
/* Exported for the tests: CRT of k residues into little-endian 32-bit limbs. */
int or_crt(const u64* x, const u64* p, u32 k, u32* limbs_out, u32 nlimbs) {
  u64 inv[OR_MAXA * OR_MAXA];
  if (k == 0 || k > OR_MAXA) return OR_E_PARAM;
  for (u32 i = 0; i < k; i++)
    for (u32 j = 0; j < k; j++) inv[i * k + j] = (i == j) ? 1 : invmod(p[j] % p[i], p[i]);
  bn X;
  crt_garner(x, p, k, inv, &X);
  memset(limbs_out, 0, sizeof(u32) * nlimbs);
  for (int i = 0; i < X.n && i < (int)nlimbs; i++) limbs_out[i] = X.d[i];
  return 0;
}

/* ------------------------------------------------------------------ */
/* context: the BFV parameters of one setup                            */
/* ------------------------------------------------------------------ */
typedef struct {
  u32 N, lg, k, na;
  u64 t, psit;
  u64 q[OR_MAXK];
  u64 qa[OR_MAXA];
  ntt_tab tq[OR_MAXK], ta[OR_MAXA], tt;
  u64 invq[OR_MAXK * OR_MAXK];
  u64 inva[OR_MAXA * OR_MAXA];
  bn Q, Qhalf;   /* Q and (Q-1)/2 */
  bn PA, PAhalf; /* product of auxiliary primes and (PA-1)/2 */
  bn Qdt;        /* floor(Q / t) */
  u64 Qmt;       /* Q mod t */
} or_ctx;

void or_free(or_ctx* c) {
  if (!c) return;
  for (u32 i = 0; i < c->k; i++) tab_free(&c->tq[i]);
  for (u32 i = 0; i < c->na; i++) tab_free(&c->ta[i]);
  tab_free(&c->tt);
  free(c);
}

/* Setup: primes per the prime-search reading (largest below 2^bits, = 1 mod
 * 2N, in the order given), minimal roots, and enough auxiliary 61-bit
 * primes for exact integer products of two centred mod-Q polynomials. */
or_ctx* or_create(u32 N, u64 t, u32 k, const unsigned char* bits) {
  if (N < 2 || (N & (N - 1)) || k == 0 || k > OR_MAXK) return NULL;
  if ((t - 1) % (2ULL * N) != 0 || !or_is_prime(t)) return NULL;
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  if (!c) return NULL;
  c->N = N; c->lg = ilog2(N); c->k = k; c->t = t;
  for (u32 i = 0; i < k; i++) {
    c->q[i] = or_find_prime(bits[i], N, c->q, i);
    if (!c->q[i] || bits[i] > 60) { c->k = i; or_free(c); return NULL; }
  }
  c->psit = or_min_root(t, N);
  tab_init(&c->tt, t, N, c->psit);
  for (u32 i = 0; i < k; i++) tab_init(&c->tq[i], c->q[i], N, or_min_root(c->q[i], N));
  bn_set_u64(&c->Q, 1);
  for (u32 i = 0; i < k; i++) bn_mul_u64(&c->Q, &c->Q, c->q[i]);
  { bn one; bn_set_u64(&one, 1); bn_sub(&c->Qhalf, &c->Q, &one); }
  bn_divmod(&c->Qhalf, NULL, &c->Qhalf, &(bn){.d = {2}, .n = 1});
  for (u32 i = 0; i < k; i++)
    for (u32 j = 0; j < k; j++) c->invq[i * k + j] = (i == j) ? 1 : invmod(c->q[j] % c->q[i], c->q[i]);
  /* auxiliary primes: product must exceed 4 * G * N * Q^2 (two products of
   * centred values summed, both signs, over up to G = OR_MAX_GROUP layers
   * when the rounding is deferred to the group), times N * t / 2 for the
   * product with a value plaintext (centred coefficients, |v| <= t/2) */
  double need = log2((double)N) + 2.0 * bn_log2(&c->Q) + 3.0 + log2((double)OR_MAX_GROUP) +
                log2((double)N * (double)t), have = 0;
  c->na = 0;
  while (have < need) {
    if (c->na >= OR_MAXA) { or_free(c); return NULL; }
    u64 p = or_find_prime(61, N, c->qa, c->na);
    c->qa[c->na] = p;
    tab_init(&c->ta[c->na], p, N, or_min_root(p, N));
    c->na++;
    have += log2((double)p);
  }
  bn_set_u64(&c->PA, 1);
  for (u32 i = 0; i < c->na; i++) bn_mul_u64(&c->PA, &c->PA, c->qa[i]);
  { bn one; bn_set_u64(&one, 1); bn_sub(&c->PAhalf, &c->PA, &one); }
  bn_divmod(&c->PAhalf, NULL, &c->PAhalf, &(bn){.d = {2}, .n = 1});
  for (u32 i = 0; i < c->na; i++)
    for (u32 j = 0; j < c->na; j++) c->inva[i * c->na + j] = (i == j) ? 1 : invmod(c->qa[j] % c->qa[i], c->qa[i]);
  c->Qmt = bn_div_u64(&c->Qdt, &c->Q, t);
  return c;
}
void or_info(const or_ctx* c, u64* q, u64* psi, u64* t_psi, u32* na, u64* qa) {
  for (u32 i = 0; i < c->k; i++) { q[i] = c->q[i]; psi[i] = c->tq[i].psi; }
  *t_psi = c->psit;
  *na = c->na;
  for (u32 i = 0; i < c->na; i++) qa[i] = c->qa[i];
}
/* log2 of Q */
double or_log2_q(const or_ctx* c) { return bn_log2(&c->Q); }

/* centred CRT over the ciphertext primes: residues -> X in (-Q/2, Q/2] */
static void lift_q(const or_ctx* c, const u64* x, sbn* X) {
  crt_garner(x, c->q, c->k, c->invq, &X->m);
  X->neg = 0;
  if (bn_cmp(&X->m, &c->Qhalf) > 0) { bn_sub(&X->m, &c->Q, &X->m); X->neg = 1; }
}
/* floor division of a signed integer by a positive big integer */
static void sbn_floordiv(sbn* y, const sbn* a, const bn* d) {
  bn qq, rr;
  bn_divmod(&qq, &rr, &a->m, d);
  if (!a->neg) { y->m = qq; y->neg = 0; return; }
  if (rr.n) bn_add_u64(&qq, &qq, 1);
  y->m = qq;
  y->neg = qq.n != 0;
}
/* round(Q * v / t) mod q_i for v in [0, t): FV's scaled message (t odd, so
 * round(a/t) = floor((a + (t-1)/2) / t)). */
static void delta_m(const or_ctx* c, u64 v, u64* out /* k residues */) {
  bn a, y;
  bn_mul_u64(&a, &c->Q, v);
  bn_add_u64(&a, &a, (c->t - 1) / 2);
  bn_div_u64(&y, &a, c->t);
  for (u32 i = 0; i < c->k; i++) out[i] = bn_mod_u64(&y, c->q[i]);
}

/* ------------------------------------------------------------------ */
/* batch encoding mod t: slot s holds m(psi_t^(2s+1))                   */
/* ------------------------------------------------------------------ */
/* slots -> coefficients of m in [0, t) */
void or_encode(const or_ctx* c, const u32* slots, u32* m) {
  u32 N = c->N;
  u64* a = (u64*)malloc(sizeof(u64) * N);
  for (u32 i = 0; i < N; i++) a[i] = slots[brev(i, c->lg)] % c->t;
  ntt_inv(a, N, &c->tt);
  for (u32 i = 0; i < N; i++) m[i] = (u32)a[i];
  free(a);
}
/* coefficients -> slots */
void or_decode(const or_ctx* c, const u32* m, u32* slots) {
  u32 N = c->N;
  u64* a = (u64*)malloc(sizeof(u64) * N);
  for (u32 i = 0; i < N; i++) a[i] = m[i] % c->t;
  ntt_fwd(a, N, &c->tt);
  for (u32 s = 0; s < N; s++) slots[s] = (u32)a[brev(s, c->lg)];
  free(a);
}

/* ------------------------------------------------------------------ */
/* constant-weight code (Eq. 1; combinatorial number system mapping)    */
/* ------------------------------------------------------------------ */
/* C(n, r) saturating at 2^63 */
u64 or_binom(u64 n, u64 r) {
  if (r > n) return 0;
  u128 v = 1;
  for (u64 i = 1; i <= r; i++) {
    v = v * (n - r + i) / i;
    if (v >= ((u128)1 << 63)) return 1ULL << 63;
  }
  return (u64)v;
}
/* Eq. 1: smallest ell with C(ell, h) >= 2^lambda_bar */
u32 or_code_length(u32 lambda_bar, u32 h) {
  u128 need = (u128)1 << lambda_bar;
  for (u32 ell = h; ell < 1000000; ell++)
    if ((u128)or_binom(ell, h) >= need) return ell;
  return 0;
}
/* CW-Encode: v in [0, C(ell,h)) -> positions c_1 < ... < c_h with
 * v = sum_r C(c_r, r) (colex rank).  pos[r-1] = c_r. */
int or_cw_encode(u64 v, u32 ell, u32 h, uint16_t* pos) {
  if (v >= or_binom(ell, h)) return OR_E_PARAM;
  u64 c = ell;
  for (u32 r = h; r >= 1; r--) {
    while (or_binom(c, r) > v) c--;
    pos[r - 1] = (uint16_t)c;
    v -= or_binom(c, r);
    if (r == 1) break;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* hashing: H0 to lambda bits, permutation-based hashing, 3 bin hashes   */
/* ------------------------------------------------------------------ */
static u64 hkey(u64 hash_key, u32 i) { return or_mix64(hash_key + (u64)(i + 1) * GOLDEN); }
/* x -> (x_L, bins[0..2]) with lambda = lambda_bar + logb */
void or_hash_item(u64 hash_key, u32 lambda_bar, u32 logb, u64 x, u64* xL, u32* bins) {
  u32 lam = lambda_bar + logb;
  u64 hx = or_mix64(x ^ hkey(hash_key, 0));
  if (lam < 64) hx &= (1ULL << lam) - 1;
  u64 xh = hx >> lambda_bar;
  *xL = hx & ((1ULL << lambda_bar) - 1);
  for (u32 i = 1; i <= 3; i++)
    bins[i - 1] = (u32)(xh ^ (or_mix64(*xL ^ hkey(hash_key, i)) & ((1ULL << logb) - 1)));
}
/* Client cuckoo hashing without stash: insert at H_1; an evicted item that
 * sat at H_i moves to H_{i+1 mod 3}; more than 1000 evictions during one
 * insertion is a failure. table_val[b] = x_L or OR_DUMMY. */
/* Client cuckoo hashing with bins of gamma slots (Section 4: the client's
 * maximum bin load gamma; gamma = 1 is the paper's evaluation, Section 7).
 * Items go in input order to the first free slot of their current bin,
 * starting at H_1; when that bin is full, the occupant of slot
 * (evictions of this insertion so far) mod gamma is evicted and moves to
 * its next hash function (H_{i+1 mod 3}); more than 1000 evictions in one
 * insertion is a failure.  table_val[bin*gamma + slot] (x_L or the dummy);
 * bin_of_item[u] = bin*gamma + slot. */
int or_cuckoo_g(u64 hash_key, u32 lambda_bar, u32 logb, u32 gamma, const u64* items, u32 m, u64* table_val,
                int32_t* bin_of_item) {
  u32 b = 1u << logb;
  if (gamma < 1) return OR_E_PARAM;
  size_t cells = (size_t)b * gamma;
  int32_t* occ = (int32_t*)malloc(sizeof(int32_t) * cells); /* item index or -1, [bin][slot] */
  u32* occ_h = (u32*)malloc(sizeof(u32) * cells);
  u32* load = (u32*)calloc(b, sizeof(u32));
  u64* xl = (u64*)malloc(sizeof(u64) * (m ? m : 1));
  u32* bins = (u32*)malloc(sizeof(u32) * 3 * (m ? m : 1));
  for (size_t i = 0; i < cells; i++) occ[i] = -1;
  for (u32 u = 0; u < m; u++) or_hash_item(hash_key, lambda_bar, logb, items[u], &xl[u], &bins[3 * u]);
  int rc = OR_OK;
  for (u32 u = 0; u < m && rc == OR_OK; u++) {
    int32_t cur = (int32_t)u;
    u32 hi = 0, ev = 0;
    for (;;) {
      u32 bin = bins[3 * cur + hi];
      if (load[bin] < gamma) {
        size_t c = (size_t)bin * gamma + load[bin]++;
        occ[c] = cur;
        occ_h[c] = hi;
        break;
      }
      size_t c = (size_t)bin * gamma + ev % gamma;
      int32_t old = occ[c];
      u32 oh = occ_h[c];
      occ[c] = cur; occ_h[c] = hi;
      cur = old; hi = (oh + 1) % 3;
      if (++ev > 1000) { rc = OR_E_CUCKOO_FAIL; break; }
    }
  }
  if (rc == OR_OK) {
    for (size_t i = 0; i < cells; i++) table_val[i] = occ[i] < 0 ? OR_DUMMY : xl[occ[i]];
    for (size_t i = 0; i < cells; i++) if (occ[i] >= 0) bin_of_item[occ[i]] = (int32_t)i;
  }
  free(occ); free(occ_h); free(load); free(xl); free(bins);
  return rc;
}
/* gamma = 1 */
int or_cuckoo(u64 hash_key, u32 lambda_bar, u32 logb, const u64* items, u32 m, u64* table_val, int32_t* bin_of_item) {
  return or_cuckoo_g(hash_key, lambda_bar, logb, 1, items, m, table_val, bin_of_item);
}
/* Server simple hashing (App. Alg 7, server side): every item goes into
 * each distinct bin among its three; an x_L already present in a bin is
 * not stored twice (the first arrival stays); layer = order of arrival in
 * the bin; dummies pad to mu.  T[layer*b + bin].  More than mu entries in a
 * bin is a failure.  Arrivals are bucketed by bin in arrival order, and
 * each bin's duplicates are found by sorting its (x_L, arrival) pairs. */
typedef struct { u64 xl; u64 pos; } or_arrival;
static int cmp_arrival(const void* a, const void* b) {
  const or_arrival *x = (const or_arrival*)a, *y = (const or_arrival*)b;
  if (x->xl != y->xl) return x->xl < y->xl ? -1 : 1;
  return x->pos < y->pos ? -1 : (x->pos > y->pos);
}
int or_simple_hash_values(u64 hash_key, u32 lambda_bar, u32 logb, const u64* items, const u32* values, u64 n,
                          u32 mu, u64* T, u32* V, u32* max_load);
int or_simple_hash(u64 hash_key, u32 lambda_bar, u32 logb, const u64* items, u64 n, u32 mu, u64* T, u32* max_load) {
  return or_simple_hash_values(hash_key, lambda_bar, logb, items, NULL, n, mu, T, NULL, max_load);
}
/* The same table plus V[mu][b]: the value of the item stored at each
 * (layer, bin) (labelled PSI / PSI-Sum, Algorithms 4-5), 0 for dummies.
 * values may be NULL (then V is all zero); V may be NULL. */
int or_simple_hash_values(u64 hash_key, u32 lambda_bar, u32 logb, const u64* items, const u32* values, u64 n,
                          u32 mu, u64* T, u32* V, u32* max_load) {
  u32 b = 1u << logb;
  u64 cap = 3 * n + 1;
  u32* abin = (u32*)malloc(sizeof(u32) * cap);
  u64* axl = (u64*)malloc(sizeof(u64) * cap);
  u64* aown = (u64*)malloc(sizeof(u64) * cap); /* item of each arrival */
  u64 na = 0;
  for (u64 u = 0; u < n; u++) {
    u64 xL;
    u32 bins[3];
    or_hash_item(hash_key, lambda_bar, logb, items[u], &xL, bins);
    for (u32 i = 0; i < 3; i++) {
      int dup_bin = 0;
      for (u32 j = 0; j < i; j++) dup_bin |= (bins[j] == bins[i]);
      if (dup_bin) continue;
      abin[na] = bins[i];
      axl[na] = xL;
      aown[na] = u;
      na++;
    }
  }
  /* stable bucketing by bin */
  u64* start = (u64*)calloc((u64)b + 1, sizeof(u64));
  for (u64 e = 0; e < na; e++) start[abin[e] + 1]++;
  for (u32 i = 0; i < b; i++) start[i + 1] += start[i];
  u64* fill = (u64*)malloc(sizeof(u64) * ((u64)b + 1));
  memcpy(fill, start, sizeof(u64) * ((u64)b + 1));
  u64* order = (u64*)malloc(sizeof(u64) * (na ? na : 1));
  for (u64 e = 0; e < na; e++) order[fill[abin[e]]++] = e;
  for (u64 i = 0; i < (u64)mu * b; i++) T[i] = OR_DUMMY;
  if (V) memset(V, 0, sizeof(u32) * (u64)mu * b);
  u32 mx = 0;
  or_arrival* tmp = (or_arrival*)malloc(sizeof(or_arrival) * (na ? na : 1));
  char* dup = (char*)calloc(na ? na : 1, 1);
  for (u32 bin = 0; bin < b; bin++) {
    u64 s0 = start[bin], len = start[bin + 1] - s0;
    for (u64 r = 0; r < len; r++) {
      tmp[r].xl = axl[order[s0 + r]];
      tmp[r].pos = r;
    }
    qsort(tmp, len, sizeof(or_arrival), cmp_arrival);
    for (u64 r = 1; r < len; r++)
      if (tmp[r].xl == tmp[r - 1].xl) dup[s0 + tmp[r].pos] = 1;
    u32 layer = 0;
    for (u64 r = 0; r < len; r++) {
      if (dup[s0 + r]) continue;
      if (layer < mu) {
        T[(u64)layer * b + bin] = axl[order[s0 + r]];
        if (V && values) V[(u64)layer * b + bin] = values[aown[order[s0 + r]]];
      }
      layer++;
    }
    if (layer > mx) mx = layer;
  }
  if (max_load) *max_load = mx;
  free(abin); free(axl); free(aown); free(start); free(fill); free(order); free(tmp); free(dup);
  return mx > mu ? OR_E_BIN_OVERFLOW : OR_OK;
}

/* ------------------------------------------------------------------ */
/* keys, encryption, decryption (FV; symmetric encryption with sk_c)    */
/* ------------------------------------------------------------------ */
/* s: uniform ternary coefficients; rlk_i = (-a_i s + e_i + g_i s^2, a_i)
 * with g_i = (Q/q_i) * [(Q/q_i)^-1]_{q_i}; layout rlk[i][comp][prime][N],
 * coefficient form. */
int or_keygen(const or_ctx* c, u64 seed, int8_t* s, u64* rlk) {
  u32 N = c->N, k = c->k;
  for (u32 n = 0; n < N; n++) s[n] = (int8_t)((int)or_sample_mod(seed, or_stream(ST_SK, 0, 0), n, 3) - 1);
  /* s^2 over the integers (schoolbook negacyclic convolution) */
  i64* s2 = (i64*)calloc(N, sizeof(i64));
  for (u32 a = 0; a < N; a++) {
    if (!s[a]) continue;
    for (u32 b2 = 0; b2 < N; b2++) {
      i64 p = (i64)s[a] * s[b2];
      u32 d = a + b2;
      if (d >= N) s2[d - N] -= p; else s2[d] += p;
    }
  }
  u64 *as = (u64*)malloc(sizeof(u64) * N), *sq = (u64*)malloc(sizeof(u64) * N), *tmp = (u64*)malloc(sizeof(u64) * N);
  u64* ai = (u64*)malloc(sizeof(u64) * N);
  for (u32 i = 0; i < k; i++) {
    /* g_i mod q_j from the definition */
    bn Qi, gi;
    bn_set_u64(&Qi, 1);
    for (u32 j = 0; j < k; j++) if (j != i) bn_mul_u64(&Qi, &Qi, c->q[j]);
    u64 inv = invmod(bn_mod_u64(&Qi, c->q[i]), c->q[i]);
    bn_mul_u64(&gi, &Qi, inv);
    for (u32 j = 0; j < k; j++) {
      u64 q = c->q[j];
      u64 g = bn_mod_u64(&gi, q);
      for (u32 n = 0; n < N; n++) {
        ai[n] = or_sample_mod(seed, or_stream(ST_RLK_A, i, j), n, q);
        sq[n] = smod(s[n], q);
      }
      ring_mul(ai, sq, as, N, &c->tq[j], tmp);
      u64* r0 = rlk + (((u64)i * 2 + 0) * k + j) * N;
      u64* r1 = rlk + (((u64)i * 2 + 1) * k + j) * N;
      for (u32 n = 0; n < N; n++) {
        i64 e = or_sample_cbd(seed, or_stream(ST_RLK_E, i, 0), n);
        u64 v = submod(smod(e, q), as[n], q);
        v = addmod(v, mulmod(g, smod(s2[n], q), q), q);
        r0[n] = v;
        r1[n] = ai[n];
      }
    }
  }
  free(s2); free(as); free(sq); free(tmp); free(ai);
  return 0;
}
/* Symmetric FV encryption of `count` plaintexts m[j][N] (coefficients in
 * [0,t)): c1 = a, c0 = -a*s + e + round(Q*m/t).  a is uniform per residue,
 * e is centred binomial; ciphertext j draws from streams indexed by j. */
int or_encrypt(const or_ctx* c, const int8_t* s, const u32* m, u32 count, u64 seed, u64* cts) {
  u32 N = c->N, k = c->k;
  u64 *a = (u64*)malloc(sizeof(u64) * N), *sq = (u64*)malloc(sizeof(u64) * N);
  u64 *as = (u64*)malloc(sizeof(u64) * N), *tmp = (u64*)malloc(sizeof(u64) * N);
  u64* dm = (u64*)malloc(sizeof(u64) * N * k);
  int* e = (int*)malloc(sizeof(int) * N);
  for (u32 j = 0; j < count; j++) {
    for (u32 n = 0; n < N; n++) {
      e[n] = or_sample_cbd(seed, or_stream(ST_ENC_E, j, 0), n);
      delta_m(c, m[(u64)j * N + n], dm + (u64)n * k);
    }
    for (u32 p = 0; p < k; p++) {
      u64 q = c->q[p];
      for (u32 n = 0; n < N; n++) {
        a[n] = or_sample_mod(seed, or_stream(ST_ENC_A, j, p), n, q);
        sq[n] = smod(s[n], q);
      }
      ring_mul(a, sq, as, N, &c->tq[p], tmp);
      u64* c0 = cts + (((u64)j * 2 + 0) * k + p) * N;
      u64* c1 = cts + (((u64)j * 2 + 1) * k + p) * N;
      for (u32 n = 0; n < N; n++) {
        c0[n] = addmod(submod(smod(e[n], q), as[n], q), dm[(u64)n * k + p], q);
        c1[n] = a[n];
      }
    }
  }
  free(a); free(sq); free(as); free(tmp); free(dm); free(e);
  return 0;
}
/* FV decryption: z = [c0 + c1*s]_Q (centred), m = [round(t*z/Q)]_t, then
 * slots.  Noise budget = log2(Q) - log2(2*max|[t*z]_Q|) (centred), which is
 * positive exactly when decryption is correct. */
/* Decryption of a ciphertext over the first r primes, modulus
 * Q_r = q_0 ... q_{r-1} (r = k: the full modulus; r < k: a response after
 * modulus switching): z = [c0 + c1 s]_{Q_r} centred, m = [round(t z / Q_r)]_t,
 * slots = Decode(m); budget = log2 Q_r - 1 - log2 max |[t z]_{Q_r}| (centred),
 * positive exactly when the decryption is correct. */
int or_decrypt_primes(const or_ctx* c, const int8_t* s, const u64* ct, u32 r, u32* slots, double* budget) {
  u32 N = c->N;
  if (r == 0 || r > c->k) return OR_E_PARAM;
  u64* z = (u64*)malloc(sizeof(u64) * N * r);
  u64 *sq = (u64*)malloc(sizeof(u64) * N), *tmp = (u64*)malloc(sizeof(u64) * N), *prod = (u64*)malloc(sizeof(u64) * N);
  for (u32 p = 0; p < r; p++) {
    u64 q = c->q[p];
    for (u32 n = 0; n < N; n++) sq[n] = smod(s[n], q);
    ring_mul(ct + ((u64)1 * r + p) * N, sq, prod, N, &c->tq[p], tmp);
    for (u32 n = 0; n < N; n++) z[(u64)n * r + p] = addmod(ct[(u64)p * N + n], prod[n], q);
  }
  /* Q_r, (Q_r - 1)/2 and the Garner inverses of the first r primes */
  bn Qr, Qrh, one;
  bn_set_u64(&Qr, 1);
  for (u32 p = 0; p < r; p++) bn_mul_u64(&Qr, &Qr, c->q[p]);
  bn_set_u64(&one, 1);
  bn_sub(&Qrh, &Qr, &one);
  bn_divmod(&Qrh, NULL, &Qrh, &(bn){.d = {2}, .n = 1});
  u64 inv[OR_MAXK * OR_MAXK];
  for (u32 i = 0; i < r; i++)
    for (u32 j = 0; j < r; j++) inv[i * r + j] = (i == j) ? 1 : invmod(c->q[j] % c->q[i], c->q[i]);
  u32* mm = (u32*)malloc(sizeof(u32) * N);
  bn maxr;
  bn_zero(&maxr);
  for (u32 n = 0; n < N; n++) {
    sbn Z, num, y;
    crt_garner(z + (u64)n * r, c->q, r, inv, &Z.m);
    Z.neg = 0;
    if (bn_cmp(&Z.m, &Qrh) > 0) { bn_sub(&Z.m, &Qr, &Z.m); Z.neg = 1; }
    /* m = round(t*Z/Q_r) mod t */
    bn_mul_u64(&num.m, &Z.m, c->t);
    num.neg = Z.neg && num.m.n;
    sbn half = {Qrh, 0};
    sbn_add(&num, &num, &half);
    sbn_floordiv(&y, &num, &Qr);
    mm[n] = (u32)sbn_mod_u64(&y, c->t);
    /* [t*Z]_{Q_r} centred */
    bn tz, rr;
    bn_mul_u64(&tz, &Z.m, c->t);
    bn_divmod(NULL, &rr, &tz, &Qr);
    if (Z.neg && rr.n) bn_sub(&rr, &Qr, &rr); /* t*Z mod Q_r for negative Z */
    if (bn_cmp(&rr, &Qrh) > 0) bn_sub(&rr, &Qr, &rr);
    if (bn_cmp(&rr, &maxr) > 0) maxr = rr;
  }
  or_decode(c, mm, slots);
  if (budget) {
    if (maxr.n == 0) *budget = INFINITY;
    else *budget = bn_log2(&Qr) - 1.0 - bn_log2(&maxr);
  }
  free(z); free(sq); free(tmp); free(prod); free(mm);
  return 0;
}
int or_decrypt(const or_ctx* c, const int8_t* s, const u64* ct, u32* slots, double* budget) {
  return or_decrypt_primes(c, s, ct, c->k, slots, budget);
}

/* Modulus switching of a ciphertext to the first r primes (the response of
 * the server computation): each coefficient's centred lift c~ in
 * (-Q/2, Q/2] becomes round(c~ * Q_r / Q) = round(c~ / Q'), Q' = Q / Q_r
 * (odd, so there are no ties), reduced mod q_0 .. q_{r-1}.
 * ct: [2][k][N], out: [2][r][N], 1 <= r <= k. */
int or_mod_switch(const or_ctx* c, const u64* ct, u32 r, u64* out) {
  u32 N = c->N, k = c->k;
  if (r == 0 || r > k) return OR_E_PARAM;
  bn Qd, Qdh, one;
  bn_set_u64(&Qd, 1);
  for (u32 p = r; p < k; p++) bn_mul_u64(&Qd, &Qd, c->q[p]);
  bn_set_u64(&one, 1);
  bn_sub(&Qdh, &Qd, &one);
  bn_divmod(&Qdh, NULL, &Qdh, &(bn){.d = {2}, .n = 1});
  sbn half = {Qdh, 0};
  u64 x[OR_MAXK];
  for (u32 comp = 0; comp < 2; comp++)
    for (u32 n = 0; n < N; n++) {
      sbn X, num, y;
      for (u32 p = 0; p < k; p++) x[p] = ct[((u64)comp * k + p) * N + n];
      lift_q(c, x, &X);
      num = X;
      sbn_add(&num, &num, &half);
      sbn_floordiv(&y, &num, &Qd);
      for (u32 p = 0; p < r; p++) out[((u64)comp * r + p) * N + n] = sbn_mod_u64(&y, c->q[p]);
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* BFV homomorphic operations (FV; ciphertexts coefficient form,         */
/* layout [comp][prime][N])                                            */
/* ------------------------------------------------------------------ */
/* plaintext polynomial m (coefficients in [0,t)) -> centred lift in
 * (-t/2, t/2] reduced mod each q_i: out[prime][N] */
void or_pt_lift(const or_ctx* c, const u32* m, u64* out) {
  for (u32 p = 0; p < c->k; p++)
    for (u32 n = 0; n < c->N; n++) {
      i64 v = (i64)m[n];
      if (v > (i64)(c->t / 2)) v -= (i64)c->t;
      out[(u64)p * c->N + n] = smod(v, c->q[p]);
    }
}
/* ct x pt: each component times the lifted plaintext, in R_Q */
void or_ct_mul_pt(const or_ctx* c, const u64* ct, const u32* m, u64* out) {
  u32 N = c->N, k = c->k;
  u64* pl = (u64*)malloc(sizeof(u64) * N * k);
  u64* tmp = (u64*)malloc(sizeof(u64) * N);
  or_pt_lift(c, m, pl);
  for (u32 comp = 0; comp < 2; comp++)
    for (u32 p = 0; p < k; p++)
      ring_mul(ct + ((u64)comp * k + p) * N, pl + (u64)p * N, out + ((u64)comp * k + p) * N, N, &c->tq[p], tmp);
  free(pl); free(tmp);
}
/* out = a + z*b over ncomp components (z a small signed integer) */
void or_ct_axpy(const or_ctx* c, const u64* a, i64 z, const u64* b, u32 ncomp, u64* out) {
  for (u32 comp = 0; comp < ncomp; comp++)
    for (u32 p = 0; p < c->k; p++) {
      u64 q = c->q[p], zq = smod(z, q);
      for (u32 n = 0; n < c->N; n++) {
        u64 i = ((u64)comp * c->k + p) * c->N + n;
        out[i] = addmod(a[i], mulmod(zq, b[i], q), q);
      }
    }
}
/* ct <- z*ct in place (z small signed integer) */
void or_ct_scale(const or_ctx* c, u64* ct, i64 z, u32 ncomp) {
  for (u32 comp = 0; comp < ncomp; comp++)
    for (u32 p = 0; p < c->k; p++) {
      u64 q = c->q[p], zq = smod(z, q);
      for (u32 n = 0; n < c->N; n++) {
        u64 i = ((u64)comp * c->k + p) * c->N + n;
        ct[i] = mulmod(zq, ct[i], q);
      }
    }
}
/* plaintext constant v (all slots) added: c0[0] += round(Q*[v]_t/t) */
void or_ct_add_const(const or_ctx* c, u64* ct, i64 v) {
  u64 d[OR_MAXK];
  delta_m(c, smod(v, c->t), d);
  for (u32 p = 0; p < c->k; p++) ct[(u64)p * c->N] = addmod(ct[(u64)p * c->N], d[p], c->q[p]);
}
/* FV multiplication without relinearisation:
 * (d0,d1,d2) = round(t/Q * (a0 b0, a0 b1 + a1 b0, a1 b1)) over Z[X]/(X^N+1)
 * with a, b the centred lifts in (-Q/2, Q/2], then reduced mod Q.  The
 * integer products are computed exactly: residues mod auxiliary NTT primes
 * whose product exceeds the bound, CRT back to big integers. */

/* The exact integer tensor of a and b as residues mod the auxiliary
 * primes, added into T[3][na][N] (T starts at zero for a single product). */
static int ct_tensor_aux(const or_ctx* c, const u64* a, const u64* b, u64* T) {
  u32 N = c->N, k = c->k, na = c->na;
  u64* A = (u64*)malloc(sizeof(u64) * 4 * na * N); /* [a0,a1,b0,b1][aux][N] */
  u64* tmp = (u64*)malloc(sizeof(u64) * N);
  u64* prod = (u64*)malloc(sizeof(u64) * N);
  if (!A || !tmp || !prod) { free(A); free(tmp); free(prod); return OR_E_NOMEM; }
  const u64* src[4] = {a, a + (u64)k * N, b, b + (u64)k * N};
  u64 x[OR_MAXK];
  for (u32 s = 0; s < 4; s++)
    for (u32 n = 0; n < N; n++) {
      sbn X;
      for (u32 p = 0; p < k; p++) x[p] = src[s][(u64)p * N + n];
      lift_q(c, x, &X);
      for (u32 j = 0; j < na; j++) A[((u64)s * na + j) * N + n] = sbn_mod_u64(&X, c->qa[j]);
    }
  /* (component, index of the a factor, index of the b factor):
   * d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 */
  static const int terms[4][3] = {{0, 0, 2}, {1, 0, 3}, {1, 1, 2}, {2, 1, 3}};
  for (u32 j = 0; j < na; j++) {
    u64 qa = c->qa[j];
    for (int ti = 0; ti < 4; ti++) {
      const u64* x0 = A + ((u64)terms[ti][1] * na + j) * N;
      const u64* y0 = A + ((u64)terms[ti][2] * na + j) * N;
      u64* dst = T + ((u64)terms[ti][0] * na + j) * N;
      ring_mul(x0, y0, prod, N, &c->ta[j], tmp);
      for (u32 n = 0; n < N; n++) dst[n] = addmod(dst[n], prod[n], qa);
    }
  }
  free(A); free(tmp); free(prod);
  return 0;
}
/* out[3][k][N] = round(t * X / Q) mod Q for the integers X whose residues
 * mod the auxiliary primes are T[3][na][N], centred in (-PA/2, PA/2]. */
static void ct_round_aux(const or_ctx* c, const u64* T, u64* out) {
  u32 N = c->N, k = c->k, na = c->na;
  u64 xa[OR_MAXA];
  sbn half = {c->Qhalf, 0};
  for (u32 comp = 0; comp < 3; comp++)
    for (u32 n = 0; n < N; n++) {
      sbn X, num, y;
      for (u32 j = 0; j < na; j++) xa[j] = T[((u64)comp * na + j) * N + n];
      crt_garner(xa, c->qa, na, c->inva, &X.m);
      X.neg = 0;
      if (bn_cmp(&X.m, &c->PAhalf) > 0) { bn_sub(&X.m, &c->PA, &X.m); X.neg = 1; }
      bn_mul_u64(&num.m, &X.m, c->t);
      num.neg = X.neg && num.m.n;
      sbn_add(&num, &num, &half);
      sbn_floordiv(&y, &num, &c->Q); /* round(t*X/Q), Q odd */
      for (u32 p = 0; p < k; p++) out[((u64)comp * k + p) * N + n] = sbn_mod_u64(&y, c->q[p]);
    }
}
/* X[3][na][N] <- X (x) v for the plaintext v (coefficients in [0, t),
 * centred lift), exactly over the integers (residues mod the aux primes). */
static void aux_mul_plain(const or_ctx* c, u64* X, const u32* v) {
  u32 N = c->N, na = c->na;
  u64 *vl = (u64*)malloc(sizeof(u64) * N), *prod = (u64*)malloc(sizeof(u64) * N), *tmp = (u64*)malloc(sizeof(u64) * N);
  for (u32 j = 0; j < na; j++) {
    u64 qa = c->qa[j];
    for (u32 n = 0; n < N; n++) vl[n] = v[n] <= c->t / 2 ? v[n] : qa - (c->t - v[n]);
    for (u32 comp = 0; comp < 3; comp++) {
      u64* x = X + ((u64)comp * na + j) * N;
      ring_mul(x, vl, prod, N, &c->ta[j], tmp);
      memcpy(x, prod, sizeof(u64) * N);
    }
  }
  free(vl); free(prod); free(tmp);
}
int or_ct_mult(const or_ctx* c, const u64* a, const u64* b, u64* out) {
  u64* T = (u64*)calloc((u64)3 * c->na * c->N, sizeof(u64));
  if (!T) return OR_E_NOMEM;
  int rc = ct_tensor_aux(c, a, b, T);
  if (!rc) ct_round_aux(c, T, out);
  free(T);
  return rc;
}
/* Deferred rounding over n products (lazy rescaling of a sum of products):
 * out = round(t/Q * sum_i v_i (x) a_i (x) b_i) mod Q, one rounding of the
 * sum of the exact integer tensors, each times the centred lift of the
 * plaintext v_i[N] (coefficients in [0, t)) when v is not NULL.
 * a, b: [n][2][k][N]; v: [n][N] or NULL; 1 <= n <= OR_MAX_GROUP. */
int or_ct_mult_sum(const or_ctx* c, const u64* a, const u64* b, const u32* v, u32 n, u64* out) {
  if (n == 0 || n > OR_MAX_GROUP) return OR_E_PARAM;
  u64 ct2 = 2ULL * c->k * c->N, tx = 3ULL * c->na * c->N;
  u64* T = (u64*)calloc(tx, sizeof(u64));
  u64* X = (u64*)malloc(sizeof(u64) * tx);
  if (!T || !X) { free(T); free(X); return OR_E_NOMEM; }
  int rc = 0;
  for (u32 i = 0; i < n && !rc; i++) {
    memset(X, 0, sizeof(u64) * tx);
    rc = ct_tensor_aux(c, a + i * ct2, b + i * ct2, X);
    if (v) aux_mul_plain(c, X, v + (u64)i * c->N);
    for (u32 comp = 0; comp < 3; comp++)
      for (u32 j = 0; j < c->na; j++)
        for (u32 m = 0; m < c->N; m++) {
          u64 e = ((u64)comp * c->na + j) * c->N + m;
          T[e] = addmod(T[e], X[e], c->qa[j]);
        }
  }
  if (!rc) ct_round_aux(c, T, out);
  free(T); free(X);
  return rc;
}
/* Relinearisation with RNS digits (no special prime): d_i = [d2]_{q_i} in
 * [0, q_i); (c0, c1) = (d0, d1) + sum_i d_i * rlk_i. */
int or_relin(const or_ctx* c, const u64* rlk, const u64* in, u64* out) {
  u32 N = c->N, k = c->k;
  u64 *dig = (u64*)malloc(sizeof(u64) * N), *prod = (u64*)malloc(sizeof(u64) * N), *tmp = (u64*)malloc(sizeof(u64) * N);
  memcpy(out, in, sizeof(u64) * 2 * k * N);
  for (u32 i = 0; i < k; i++) {
    const u64* d2i = in + ((u64)2 * k + i) * N; /* residue of d2 mod q_i */
    for (u32 j = 0; j < k; j++) {
      u64 q = c->q[j];
      for (u32 n = 0; n < N; n++) dig[n] = d2i[n] % q;
      for (u32 comp = 0; comp < 2; comp++) {
        ring_mul(dig, rlk + (((u64)i * 2 + comp) * k + j) * N, prod, N, &c->tq[j], tmp);
        u64* o = out + ((u64)comp * k + j) * N;
        for (u32 n = 0; n < N; n++) o[n] = addmod(o[n], prod[n], q);
      }
    }
  }
  free(dig); free(prod); free(tmp);
  return 0;
}

/* ------------------------------------------------------------------ */
/* PEPSI server computation (Alg 1 inside Alg 2; cardinality per Alg 5) */
/* ------------------------------------------------------------------ */
/* CW-Encode of every entry of one table row: pos[s*h + r], dummies marked
 * with 0xFFFF in pos[s*h]. */
static void row_codewords(const u64* row, u32 N, u32 ell, u32 h, uint16_t* pos) {
  for (u32 s = 0; s < N; s++) {
    if (row[s] == OR_DUMMY) { pos[(u64)s * h] = 0xFFFF; continue; }
    or_cw_encode(row[s], ell, h, pos + (u64)s * h);
  }
}
/* slot vector of bit j of the codewords of one row (dummy -> all zeros) */
static void bit_plane(const uint16_t* pos, u32 N, u32 h, u32 j, u32* slots) {
  for (u32 s = 0; s < N; s++) {
    slots[s] = 0;
    if (pos[(u64)s * h] == 0xFFFF) continue;
    for (u32 r = 0; r < h; r++) slots[s] |= (pos[(u64)s * h + r] == j);
  }
}
/* Server plaintext pt_s[layer][j] (App. Alg 7 batching) in NTT form:
 * out[prime][N] = NTT_{q_i}(lift(Encode(bit plane j of layer))). */
void or_server_plaintext(const or_ctx* c, const u64* T, u32 ell, u32 h, u32 layer, u32 j, u64* out) {
  u32 N = c->N;
  u32 *sl = (u32*)malloc(sizeof(u32) * N), *m = (u32*)malloc(sizeof(u32) * N);
  uint16_t* pos = (uint16_t*)malloc(sizeof(uint16_t) * N * (h ? h : 1));
  row_codewords(T + (u64)layer * N, N, ell, h, pos);
  bit_plane(pos, N, h, j, sl);
  or_encode(c, sl, m);
  or_pt_lift(c, m, out);
  for (u32 p = 0; p < c->k; p++) ntt_fwd(out + (u64)p * N, N, &c->tq[p]);
  free(sl); free(m); free(pos);
}
/* Client query plaintexts: m[j][N] = Encode(bit plane j of the client
 * table row), j in [0, ell). */
void or_query_plaintexts(const or_ctx* c, const u64* Tc, u32 ell, u32 h, u32* m) {
  u32 N = c->N;
  u32* sl = (u32*)malloc(sizeof(u32) * N);
  uint16_t* pos = (uint16_t*)malloc(sizeof(uint16_t) * N * (h ? h : 1));
  row_codewords(Tc, N, ell, h, pos);
  for (u32 j = 0; j < ell; j++) {
    bit_plane(pos, N, h, j, sl);
    or_encode(c, sl, m + (u64)j * N);
  }
  free(sl); free(pos);
}

/* Arith-CW-Eq (Alg 1) on one layer, from h' (3-component buffer with d2 = 0):
 *   h=1: E = h'
 *   h=2: E = Mult(h', h' - 1)
 *   h=4: u = R(Mult(h',h')) - 3h';  E = Mult(u, u + 2)
 *   h=8: u = R(Mult(h',h')) - 7h';  w = R(Mult(u,u));
 *        E = Mult(w + 12u, w + 16u + 60)
 * which equal prod_{i<h}(h' - i); the factor 1/h! is applied once after the
 * sum over layers.  E is left without relinearisation.
 * With Xaux non-NULL (h >= 2) the last Mult is not rounded: the exact
 * integer tensor of its operands is added into Xaux[3][na][N] (residues
 * mod the auxiliary primes) instead, and E is not written. */
static int eq_circuit(const or_ctx* c, const u64* rlk, u32 h, const u64* hp /*[2][k][N]*/, u64* E /*[3][k][N]*/,
                      u64* Xaux, u32* nmult) {
  u32 N = c->N, k = c->k;
  u64 ct2 = 2ULL * k * N, ct3 = 3ULL * k * N;
  u64* buf = (u64*)calloc(8 * ct3, sizeof(u64));
  if (!buf) return OR_E_NOMEM;
  u64 *t3 = buf, *u = buf + ct3, *w = buf + 2 * ct3, *x = buf + 3 * ct3, *y = buf + 4 * ct3;
  int rc = 0;
  if (E) memset(E, 0, sizeof(u64) * ct3);
  switch (h) {
    case 1:
      memcpy(E, hp, sizeof(u64) * ct2);
      break;
    case 2:
      memcpy(x, hp, sizeof(u64) * ct2);
      or_ct_add_const(c, x, -1);
      rc = Xaux ? ct_tensor_aux(c, hp, x, Xaux) : or_ct_mult(c, hp, x, E); (*nmult)++;
      break;
    case 4:
      rc = or_ct_mult(c, hp, hp, t3); (*nmult)++;
      or_relin(c, rlk, t3, u);
      or_ct_axpy(c, u, -3, hp, 2, u);
      memcpy(x, u, sizeof(u64) * ct2);
      or_ct_add_const(c, x, 2);
      rc |= Xaux ? ct_tensor_aux(c, u, x, Xaux) : or_ct_mult(c, u, x, E); (*nmult)++;
      break;
    case 8:
      rc = or_ct_mult(c, hp, hp, t3); (*nmult)++;
      or_relin(c, rlk, t3, u);
      or_ct_axpy(c, u, -7, hp, 2, u);
      rc |= or_ct_mult(c, u, u, t3); (*nmult)++;
      or_relin(c, rlk, t3, w);
      or_ct_axpy(c, w, 12, u, 2, x);
      or_ct_axpy(c, w, 16, u, 2, y);
      or_ct_add_const(c, y, 60);
      rc |= Xaux ? ct_tensor_aux(c, x, y, Xaux) : or_ct_mult(c, x, y, E); (*nmult)++;
      break;
    default:
      rc = OR_E_PARAM;
  }
  free(buf);
  return rc;
}

/* centred representative of (h!)^-1 mod t */
static i64 inv_hfact(const or_ctx* c, u32 h) {
  u64 f = 1;
  for (u32 i = 2; i <= h; i++) f = mulmod(f, i, c->t);
  u64 z = invmod(f, c->t);
  return z > c->t / 2 ? (i64)z - (i64)c->t : (i64)z;
}

/* Alg 2 for one client batch (gamma = 1, b = N) over server layers
 * [layer0, layer0+nl):
 *   h'_{i'} = sum_j ct_c[j] (x) pt_s[i'][j];  E_{i'} = Arith-CW-Eq circuit;
 *   A = sum_{i'} E_{i'};  ct = (h!)^-1 * R(A);
 *   mode 1 (cardinality, Alg 5 with val = 1): ct += (round(Q*Encode(r)/t), 0)
 *   with r uniform in Z_t^N, r_{N-1} = -sum of the others.
 *   mode 2 (labelled PSI, Alg 4): A = sum_{i'} val_s[i'] * E_{i'}, where
 *   val_s[i'] = Encode(V[i'][.]) (centred lift) holds the value of the
 *   item stored in each bin of layer i'.
 *   mode 3 (PSI-Sum, Alg 5): as mode 2, plus the mask of mode 1.
 * cts: [ell][2][k][N] coefficient form.  T: server table [mu][N].
 * dbg_h: [nl][2][k][N] h' (coefficient form), dbg_e: [nl][3][k][N] E.
 * dbg_acc: [3][k][N] the layer sum A before relinearisation.
 * counts (optional): [0] plaintext mults, [1] ciphertext mults.
 * group: rounding of the last Mult of each layer.  group <= 1 rounds every
 * layer (E_{i'} as above).  group = G > 1 (lazy rescaling, h >= 2) splits
 * the layers, from layer0 on, into runs of G consecutive layers; the exact
 * integer tensors of a run's last Mults are summed and rounded once,
 * round(t/Q * sum X_{i'}), and the runs' results are summed mod Q into A.
 * Per-layer E words do not exist then, so dbg_e must be NULL.  In modes 2
 * and 3 a run sums val_s[i'] (x) X_{i'} (the value product taken before
 * the run's rounding); with group <= 1 val_s[i'] multiplies the rounded
 * E_{i'}, as Algorithms 4-5 write it.
 * The plaintext-times-ciphertext sums are accumulated in the NTT domain
 * and transformed back once per layer (the inverse NTT is linear). */
int or_eval(const or_ctx* c, const u64* rlk, const u64* cts, u32 ell, u32 h, const u64* T, const u32* V, u32 mu,
            u32 layer0, u32 nl, int mode, u64 mask_seed, u32 group, u64* out, u64* dbg_h, u64* dbg_e,
            u64* dbg_acc, u64* counts) {
  u32 N = c->N, k = c->k;
  if (layer0 + nl > mu || (h != 1 && h != 2 && h != 4 && h != 8)) return OR_E_PARAM;
  if (mode < 0 || mode > 3) return OR_E_PARAM;
  const int valued = mode >= 2;
  if (valued && !V) return OR_E_PARAM;
  if (group > OR_MAX_GROUP) return OR_E_PARAM;
  const int lazy = group > 1 && h > 1;
  if (lazy && dbg_e) return OR_E_PARAM;
  u64 ct2 = 2ULL * k * N, ct3 = 3ULL * k * N, ctx = 3ULL * c->na * N;
  /* query ciphertexts to NTT form */
  u64* CN = (u64*)malloc(sizeof(u64) * ell * ct2);
  if (!CN) return OR_E_NOMEM;
  memcpy(CN, cts, sizeof(u64) * ell * ct2);
#pragma omp parallel for schedule(dynamic)
  for (long jj = 0; jj < (long)ell * 2 * k; jj++) ntt_fwd(CN + (u64)jj * N, N, &c->tq[jj % k]);
  u64* Eall = (u64*)calloc((u64)(nl ? nl : 1) * (lazy ? ctx : ct3), sizeof(u64)); /* E, or X when lazy */
  u64 pm = 0, mm = 0;
  int rc = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : pm, mm) reduction(| : rc)
  for (long li = 0; li < (long)nl; li++) {
    u32 layer = layer0 + (u32)li;
    u128* acc = (u128*)calloc(ct2, sizeof(u128));
    u64* pt = (u64*)malloc(sizeof(u64) * k * N);
    u64* hp = (u64*)malloc(sizeof(u64) * ct2);
    u32 nm = 0;
    u32 *sl = (u32*)malloc(sizeof(u32) * N), *mt = (u32*)malloc(sizeof(u32) * N);
    uint16_t* pos = (uint16_t*)malloc(sizeof(uint16_t) * N * h);
    row_codewords(T + (u64)layer * N, N, ell, h, pos);
    for (u32 j = 0; j < ell; j++) {
      /* pt_s[layer][j] in NTT form (App. Alg 7 batching, then lift, NTT) */
      bit_plane(pos, N, h, j, sl);
      or_encode(c, sl, mt);
      or_pt_lift(c, mt, pt);
      for (u32 p = 0; p < k; p++) ntt_fwd(pt + (u64)p * N, N, &c->tq[p]);
      for (u32 comp = 0; comp < 2; comp++)
        for (u32 p = 0; p < k; p++)
          for (u32 n = 0; n < N; n++) {
            u64 i = ((u64)comp * k + p) * N + n;
            acc[i] += (u128)CN[(u64)j * ct2 + i] * pt[(u64)p * N + n];
            if (acc[i] >> 127) acc[i] %= c->q[p]; /* keeps the sum below 2^128 */
          }
      pm++;
    }
    for (u32 comp = 0; comp < 2; comp++)
      for (u32 p = 0; p < k; p++) {
        u64* hrow = hp + ((u64)comp * k + p) * N;
        for (u32 n = 0; n < N; n++) hrow[n] = (u64)(acc[((u64)comp * k + p) * N + n] % c->q[p]);
        ntt_inv(hrow, N, &c->tq[p]);
      }
    if (dbg_h) memcpy(dbg_h + (u64)li * ct2, hp, sizeof(u64) * ct2);
    if (lazy)
      rc |= eq_circuit(c, rlk, h, hp, NULL, Eall + (u64)li * ctx, &nm);
    else
      rc |= eq_circuit(c, rlk, h, hp, Eall + (u64)li * ct3, NULL, &nm);
    if (valued) { /* val_s[layer] (Alg 4 / 5) */
      or_encode(c, V + (u64)layer * N, mt);
      if (lazy) {
        aux_mul_plain(c, Eall + (u64)li * ctx, mt);
      } else {
        u64* E = Eall + (u64)li * ct3;
        u64* pl = (u64*)malloc(sizeof(u64) * k * N);
        u64 *prod = (u64*)malloc(sizeof(u64) * N), *tmp = (u64*)malloc(sizeof(u64) * N);
        or_pt_lift(c, mt, pl);
        for (u32 comp = 0; comp < 3; comp++)
          for (u32 p = 0; p < k; p++) {
            u64* e = E + ((u64)comp * k + p) * N;
            ring_mul(e, pl + (u64)p * N, prod, N, &c->tq[p], tmp);
            memcpy(e, prod, sizeof(u64) * N);
          }
        free(pl); free(prod); free(tmp);
      }
    }
    mm += nm;
    if (dbg_e) memcpy(dbg_e + (u64)li * ct3, Eall + (u64)li * ct3, sizeof(u64) * ct3);
    free(acc); free(pt); free(hp); free(sl); free(mt); free(pos);
  }
  if (rc) { free(CN); free(Eall); return rc; }
  /* A = sum over layers (mod Q) */
  u64* A = (u64*)calloc(ct3, sizeof(u64));
  if (lazy) {
    /* each run of `group` layers: sum the exact tensors, round once */
    u64* Xg = (u64*)malloc(sizeof(u64) * ctx);
    u64* Eg = (u64*)malloc(sizeof(u64) * ct3);
    for (u32 g0 = 0; g0 < nl; g0 += group) {
      u32 g1 = g0 + group < nl ? g0 + group : nl;
      memset(Xg, 0, sizeof(u64) * ctx);
      for (u32 li = g0; li < g1; li++)
        for (u32 comp = 0; comp < 3; comp++)
          for (u32 j = 0; j < c->na; j++)
            for (u32 n = 0; n < N; n++) {
              u64 i = ((u64)comp * c->na + j) * N + n;
              Xg[i] = addmod(Xg[i], Eall[(u64)li * ctx + i], c->qa[j]);
            }
      ct_round_aux(c, Xg, Eg);
      for (u32 comp = 0; comp < 3; comp++)
        for (u32 p = 0; p < k; p++)
          for (u32 n = 0; n < N; n++) {
            u64 i = ((u64)comp * k + p) * N + n;
            A[i] = addmod(A[i], Eg[i], c->q[p]);
          }
    }
    free(Xg); free(Eg);
  } else {
    for (u32 li = 0; li < nl; li++)
      for (u32 comp = 0; comp < 3; comp++)
        for (u32 p = 0; p < k; p++)
          for (u32 n = 0; n < N; n++) {
            u64 i = ((u64)comp * k + p) * N + n;
            A[i] = addmod(A[i], Eall[(u64)li * ct3 + i], c->q[p]);
          }
  }
  if (dbg_acc) memcpy(dbg_acc, A, sizeof(u64) * ct3);
  or_relin(c, rlk, A, out);
  or_ct_scale(c, out, inv_hfact(c, h), 2);
  if (mode == 1 || mode == 3) {
    u32 *r = (u32*)malloc(sizeof(u32) * N), *mr = (u32*)malloc(sizeof(u32) * N);
    u64 sum = 0;
    for (u32 s = 0; s + 1 < N; s++) {
      r[s] = (u32)or_sample_mod(mask_seed, or_stream(ST_MASK, 0, 0), s, c->t);
      sum = (sum + r[s]) % c->t;
    }
    r[N - 1] = (u32)((c->t - sum) % c->t);
    or_encode(c, r, mr);
    u64 d[OR_MAXK];
    for (u32 n = 0; n < N; n++) {
      delta_m(c, mr[n], d);
      for (u32 p = 0; p < k; p++) out[(u64)p * N + n] = addmod(out[(u64)p * N + n], d[p], c->q[p]);
    }
    free(r); free(mr);
  }
  if (counts) { counts[0] = pm; counts[1] = mm; }
  free(CN); free(Eall); free(A);
  return 0;
}

void or_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int or_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
