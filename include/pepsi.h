/*
 * pepsi.h -- C ABI of the GB300 (sm_103a) implementation of PEPSI's
 * server-side homomorphic evaluation (arXiv 2310.14565).
 *
 * The library evaluates Algorithm 2 ("Intersect") with the arithmetic
 * constant-weight equality operator of Algorithm 1 in RNS-BFV (FV,
 * Section 3.1), the cardinality variant of Algorithm 5, and the client
 * side of Algorithms 3 and 7 needed to produce and read the messages.
 *
 * Conventions shared by every call:
 *  - Return value: PEPSI_OK (0) or one of the error codes below.  No call
 *    aborts the process; pepsi_strerror() names a code.
 *  - Pointers: the caller owns every buffer it passes.  "host or device"
 *    means the library inspects the pointer (cudaPointerGetAttributes) and
 *    copies through the call's stream when it is host memory.  The context
 *    owns all of its device memory (keys, server tables, scratch).
 *  - Ciphertext words: residues in [0, q_i), layout [component][prime][N]
 *    (prime-major inside a component), coefficient form unless stated.
 *    A batch of ciphertexts adds a leading dimension.
 *  - Streams: `stream` is a cudaStream_t (NULL: the context's own stream).
 *    Calls with device output buffers are asynchronous on that stream;
 *    calls with host output buffers synchronise it before returning.
 *  - One context serves one evaluation at a time: calls on the same
 *    context must not overlap (they share the context's scratch memory).
 *  - Parameters the paper leaves open (prime choice, roots, hashing
 *    functions, randomness, codeword mapping, slot order) follow the
 *    readings documented with the project and implemented identically by
 *    its independent CPU oracle.
 */
#ifndef PEPSI_H
#define PEPSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
enum {
  PEPSI_OK = 0,
  PEPSI_E_PARAM = 1,        /* invalid or unsupported parameters / arguments */
  PEPSI_E_BIN_OVERFLOW = 2, /* a server bin holds more than mu items (Section 4.1) */
  PEPSI_E_CUCKOO_FAIL = 3,  /* client cuckoo insertion exceeded the eviction bound (Section 3.3) */
  PEPSI_E_NOMEM = 4,        /* device memory (HBM budget) exhausted */
  PEPSI_E_CUDA = 5,         /* a CUDA runtime call failed */
  PEPSI_E_TIMEOUT = 6,      /* a bounded device wait expired */
  PEPSI_E_NOISE = 7         /* decryption noise budget exhausted (<= 0 bits) */
};

/* Evaluation modes. */
enum {
  PEPSI_MODE_INDICATOR = 0,   /* Algorithm 2: encrypted per-bin indicator */
  PEPSI_MODE_CARDINALITY = 1, /* Algorithm 5 with val_s = 1: masked, slots sum to |X cap Y| */
  PEPSI_MODE_LABELS = 2,      /* Algorithm 4: slot of a matched client item = the server item's value
                                 (0 otherwise); needs a set loaded with values */
  PEPSI_MODE_SUM = 3          /* Algorithm 5: masked, slots sum to the matched items' values mod t;
                                 needs a set loaded with values */
};

/* pepsi_params.rescale_group: one rounding for all layers of an evaluation. */
#define PEPSI_RESCALE_ALL 0xFFFFFFFFu

typedef struct pepsi_ctx pepsi_ctx; /* opaque */

/* Parameters (Table 2 notation).  Zero means "derive". */
typedef struct {
  uint32_t N;              /* ring degree = number of bins b (power of two, 16..16384) */
  uint64_t t;              /* plaintext modulus: prime, t = 1 (mod 2N), t < 2^32 */
  uint32_t k;              /* number of ciphertext primes q_i (1..8) */
  uint8_t prime_bits[8];   /* bit size of each q_i (20..60), searched in this order */
  uint32_t h;              /* Hamming weight of the constant-weight code: 1, 2, 4 or 8 */
  uint32_t ell;            /* code length; 0 -> Eq. 1 from lambda_bar and h */
  uint32_t lambda_bar;     /* effective item bit length (Section 3.3, PBH) */
  uint32_t num_hashes;     /* cuckoo / simple hash functions: must be 3 */
  uint32_t mu;             /* server maximum bin load; 0 -> bound rule */
  uint64_t hash_key;       /* public seed of H_0..H_3 */
  uint64_t resident_bytes; /* HBM budget for resident server plaintexts: the longest
                              prefix of layers that fits stays resident, the rest is
                              regenerated per chunk at evaluation.  0: 60% of free
                              HBM at load time; UINT64_MAX: none; else a byte cap */
  uint32_t rescale_group;  /* rounding of the last ciphertext product of each layer in
                              pepsi_eval / pepsi_eval_batch.  0 or 1: every layer's product
                              is rounded, round(t/Q * X), as in textbook FV multiplication.
                              G > 1 (lazy rescaling): the exact integer products of runs of
                              G consecutive layers (from the first evaluated layer) are
                              summed in the auxiliary base and each run is rounded once,
                              round(t/Q * sum X); the result decrypts the same, its words
                              differ, and each run saves the inverse transforms and the
                              rounding of G - 1 products.  PEPSI_RESCALE_ALL: one run per
                              evaluation.  The auxiliary base is sized at setup for runs of
                              up to pepsi_info.rescale_cap layers (G itself; for
                              PEPSI_RESCALE_ALL mu, or 65536 when mu = 0); longer runs are
                              cut at the cap.  pepsi_eval_layers always rounds per layer. */
  uint32_t server_values;  /* nonzero: the auxiliary base also holds the value products of
                              the LABELS and SUM modes under lazy rescaling (log2(N t / 2)
                              more bits); with 0 those modes round per layer */
  uint32_t response_primes;/* primes r of the evaluation's response: pepsi_eval and
                              pepsi_eval_batch switch the result to q_0..q_{r-1}
                              (pepsi_mod_switch), out_ct [2][r][N]; 0 = k, no switching.
                              r = 1 gives the one-prime response (2 N 8 bytes) */
  uint32_t bins;           /* number of bins b: 0 = N; else a power of two N * B, B <= 1024.
                              The b bins form B blocks of N slots (Section 4: ceil(b/N)
                              ciphertexts per code bit): the request holds B * ell
                              ciphertexts [B][ell][2][k][N], every server layer one block of
                              plaintexts per request block, and the response B ciphertexts
                              [B][2][r][N], block j answering bins j*N .. j*N + N - 1 */
  uint32_t plaintext_bytes;/* storage of the resident server plaintexts (NTT form), bytes per
                              word: 0 or 8 = 64-bit words; 7 = the reduced value in three
                              planes of 4, 2 and 1 bytes (every q_i < 2^56, else PEPSI_E_PARAM):
                              12.5% more layers stay resident in the same budget, but the
                              multiply-accumulate runs slower on a fully resident table (its
                              unpacking costs more than the saved traffic).  Results are the
                              same either way */
  uint32_t gamma;          /* client maximum bin load (Table 2, Section 4): 0 or 1 = cuckoo
                              hashing with one item per bin (the paper's evaluation); 2..16 =
                              bins of gamma slots, so up to gamma * b client items.  The client
                              table's batch i is slot i of every bin: a request holds B * gamma
                              * ell ciphertexts [B][gamma][ell][2][k][N] and Algorithm 2
                              returns one indicator ciphertext per batch, [B][gamma][2][r][N] */
  uint32_t client_cuckoo;  /* placement of pepsi_query's cuckoo hashing (no counterpart in the
                              paper, which gives no algorithm for it): 0 = on the host, items
                              inserted in order with eviction chains (the placement the oracle
                              computes); 1 = on the device, in parallel rounds: every unplaced
                              item claims its current candidate bin, the smallest claiming item
                              takes a free slot of the bin or evicts the occupant of slot
                              (evictions mod gamma), which moves to its next candidate bin, and
                              the other claimants move to theirs; at most 1000 rounds.  Both
                              are deterministic valid placements (every item in one of its three
                              candidate bins, at most gamma per bin); they differ in which */
} pepsi_params;

/* Derived values of a context (for callers and tests). */
typedef struct {
  uint32_t N, k, kb, ell, h, mu, lambda_bar, logb;
  uint64_t t;
  uint64_t q[8];        /* ciphertext primes */
  uint64_t psi[8];      /* minimal primitive 2N-th roots of the q_i */
  uint64_t psi_t;       /* minimal primitive 2N-th root mod t */
  uint64_t b_primes[12];/* auxiliary base B used for exact multiplication */
  double log2_q;
  uint32_t rescale_group;/* rescale_group as given (0 and 1 both mean per layer) */
  uint32_t rescale_cap;  /* most layers one rounding may cover (1: per-layer rounding only) */
  uint32_t response_primes; /* primes of the evaluation's response (k: not switched) */
  uint32_t bins, blocks;     /* b = blocks * N bins */
  uint32_t plaintext_bytes;  /* 7 or 8: storage of the resident server plaintexts per word */
  uint32_t gamma;            /* client maximum bin load: client batches per block */
} pepsi_info;

/* Setup (Section 4, parameters of Tables 2-3): derives ell (Eq. 1), the
 * primes (largest below 2^bits with q = 1 mod 2N), the NTT tables and the
 * auxiliary base; samples the secret key s (uniform ternary) and the
 * relinearisation keys rlk_i = (-a_i s + e_i + g_i s^2, a_i) from key_seed,
 * all on the device.  *out receives the context; destroy with
 * pepsi_destroy().  Errors: PEPSI_E_PARAM, PEPSI_E_NOMEM, PEPSI_E_CUDA. */
int pepsi_setup(const pepsi_params* params, uint64_t key_seed, pepsi_ctx** out);

/* Parameter selection, host only (Section 6.1).  Request size of a query:
 * ceil(bins / N) * ell * N * log2 q bits, with ell = Eq. 1 (the smallest
 * code length with C(ell, h) >= 2^lambda_bar) and (log2 N, log2 q) the
 * smallest parameter set for Hamming weight h (Table 3: h = 1, 2, 3-4,
 * 5-8, 9-16, 17-32, 33-64).  ell, log2_n, log2_q may be NULL.  Errors:
 * PEPSI_E_PARAM for h outside 1..64, lambda_bar outside 1..62, bins = 0. */
int pepsi_request_bits(uint32_t lambda_bar, uint32_t h, uint64_t bins, double* bits, uint64_t* ell,
                       uint32_t* log2_n, uint32_t* log2_q);

/* The communication-optimal Hamming weight (Section 6.1): the h in
 * 1..h_max minimising pepsi_request_bits, a tie going to the smaller h
 * (less computation).  Host only.  Errors: PEPSI_E_PARAM. */
int pepsi_comm_optimal_h(uint32_t lambda_bar, uint64_t bins, uint32_t h_max, uint32_t* h);

/* Fill *info with the context's derived parameters. */
int pepsi_get_info(const pepsi_ctx* ctx, pepsi_info* info);

/* Set the rounding run length of later evaluations on this context, with
 * the meaning of pepsi_params.rescale_group (1: per-layer rounding; G > 1
 * or PEPSI_RESCALE_ALL: lazy rescaling).  Runs stay cut at the
 * rescale_cap fixed at setup, so every value is accepted and the result
 * stays exact.  Errors: PEPSI_E_PARAM for a null context. */
int pepsi_set_rescale_group(pepsi_ctx* ctx, uint32_t rescale_group);

/* Evaluation schedule of a context (no counterpart in the paper): how an
 * evaluation is split into launches, never what it computes.  Every field
 * leaves the result words unchanged. */
typedef struct {
  uint32_t chunk;       /* layers per circuit chunk, 1..4096 (default 64, or the
                           PEPSI_CHUNK environment variable at setup); n layers run in
                           ceil(n / chunk) chunks of equal size (within one layer), so
                           526 layers at chunk 256 run as 176, 176 and 174.  Larger chunks
                           fill the GPU with more blocks per launch and need more
                           scratch (about 4.7 MB per layer at N = 8192, k = 4) */
  uint32_t ntt_threads; /* threads per block of the ciphertext transforms (the NTTs and
                           the kernels fused with them): 0 = the default for N (N / 8,
                           at most 512; 1024 at N = 16384), else a power of two in
                           64..1024 */
  uint32_t relin_fused; /* 1 (default): where a relinearised product only feeds the
                           affine step after it (u = R(h'^2) - 3h' and the like), the
                           key-switching sum runs on the load of the inverse NTT that
                           extends u, and the relinearised product is never stored;
                           0: it is stored, then the affine step runs */
  uint32_t batch_points;/* points per block of the multiply-accumulate that serves several
                           requests with one read of the plaintexts (pepsi_eval_batch):
                           0 = the default (32), 32 (16 layers per block) or 64 (8 layers:
                           longer copy rows, more re-reads of the request tiles) */
  uint32_t batch_groups;/* warp groups of that multiply-accumulate: 0 = the default (2),
                           1 = every thread serves all requests of the group (fewer, fuller
                           warps), 2 = two groups of warps serve half the requests each
                           (twice the warps; groups of 3 requests always run with 1) */
  uint32_t batch_requests;/* most requests that share one multiply-accumulate launch in
                           pepsi_eval_batch and in an engine step (several launches when
                           more are in flight): 0 = the default (2), else 1..4 */
} pepsi_schedule;

/* Read or set the schedule of later evaluations on this context
 * (pepsi_autotune sets it too).  Errors: PEPSI_E_PARAM for a null pointer
 * or a field out of range. */
int pepsi_get_schedule(const pepsi_ctx* ctx, pepsi_schedule* out);
int pepsi_set_schedule(pepsi_ctx* ctx, const pepsi_schedule* schedule);

/* Server preprocessing, offline (Section 4.1 and App. Alg 7, server side):
 * H_0 to lambda bits, permutation-based hashing into each of the three
 * bins of every item, de-duplication of equal x_L inside a bin, stable
 * layer order, dummies up to mu; then the NTT-form server plaintexts
 * pt_s[layer][j] are generated on the device: the layers that fit the
 * resident_bytes budget stay resident, the others are regenerated per
 * layer chunk at evaluation time.
 * items: host array of n 64-bit items.  *set_id receives the handle.
 * Errors: PEPSI_E_BIN_OVERFLOW, PEPSI_E_NOMEM, PEPSI_E_PARAM, PEPSI_E_CUDA. */
int pepsi_server_load(pepsi_ctx* ctx, const uint64_t* items, size_t n, int* set_id);

/* Server preprocessing with a value per item, for labelled PSI (Algorithm
 * 4) and PSI-Sum (Algorithm 5): as pepsi_server_load, and the value of the
 * item stored at each (layer, bin) (0 for dummies; of an x_L stored twice
 * in a bin, the first item's) becomes the value plaintext val_s[layer],
 * kept resident in NTT form over the ciphertext and auxiliary primes.
 * values: host array of n values in [0, t).  Errors: as pepsi_server_load;
 * PEPSI_E_PARAM for a value >= t. */
int pepsi_server_load_values(pepsi_ctx* ctx, const uint64_t* items, const uint32_t* values, size_t n,
                             int* set_id);

/* Copy the value table of a set loaded with values: out[mu][b] (host). */
int pepsi_server_values(pepsi_ctx* ctx, int set_id, uint32_t* out);

/* Copy the raw server table T_s of a set: out[mu][b] (host, b bins), entries are
 * x_L values or UINT64_MAX for dummies. */
int pepsi_server_table(pepsi_ctx* ctx, int set_id, uint64_t* out);

/* Copy server plaintexts pt_s[layer][j] for layers [layer0, layer0+nl) in
 * NTT form (value at psi^(2 brev(i)+1) in slot i): out[B][nl][ell][k][N] (B blocks),
 * host or device. */
int pepsi_server_plaintexts(pepsi_ctx* ctx, int set_id, uint32_t layer0, uint32_t nl, uint64_t* out,
                            void* stream);

/* Client request (App. Alg 7, client side): cuckoo hashing without stash
 * (3 hashes, eviction bound 1000) into bins of gamma slots, CW-Encode,
 * batching (batch i = slot i of every bin), symmetric FV encryption under s
 * with randomness from enc_seed (ciphertext i of the request draws from
 * stream index i).  cts: [B][gamma][ell][2][k][N] coefficient form (host or
 * device).  bin_of_item: host int32[m], bin * gamma + slot of each item
 * (the bin when gamma = 1).  Errors: PEPSI_E_CUCKOO_FAIL, PEPSI_E_PARAM. */
int pepsi_query(pepsi_ctx* ctx, const uint64_t* items, size_t m, uint64_t enc_seed, uint64_t* cts,
                int32_t* bin_of_item, void* stream);

/* Server computation (Algorithm 2; mode CARDINALITY adds Algorithm 5's
 * zero-sum mask drawn from mask_seed): for every layer i',
 * h' = sum_j ct_c[j] x pt_s[i'][j], e = prod_{i<h}(h' - i), summed over
 * layers, relinearised and multiplied by (h!)^-1 mod t.  Modes LABELS and
 * SUM weight layer i' by its value plaintext val_s[i'] (Algorithms 4-5):
 * with per-layer rounding val_s[i'] multiplies the rounded e; with lazy
 * rescaling it multiplies the exact product before the run's rounding.
 * cts: [B][gamma][ell][2][k][N] coefficient form, host or device.
 * out_ct: [B][gamma][2][r][N] coefficient form, host or device, with B
 * blocks, gamma client batches and r = pepsi_info.response_primes (k unless
 * the response is switched); ciphertext (j, i) of the response answers
 * client batch i of request block j, its mask drawn from
 * mask_seed + j * gamma + i.  With gamma > 1 the batches of a block are
 * evaluated as by pepsi_eval_batch (shared multiply-accumulates).  A host request is uploaded in two pieces of its code bits
 * (the first short), the copy of the second overlapping the first piece's
 * transform and multiply-accumulate; the words do not depend on it.  Device
 * buffers need 8-byte alignment (16-byte aligned rows take wider accesses).
 * Errors: PEPSI_E_PARAM (bad set/mode), PEPSI_E_NOMEM, PEPSI_E_CUDA. */
int pepsi_eval(pepsi_ctx* ctx, int set_id, const uint64_t* cts, int mode, uint64_t mask_seed, uint64_t* out_ct,
               void* stream);

/* Autotuning of the evaluation schedule (no counterpart in the paper):
 * evaluates the request cts ([B][ell][2][k][N], host or device) against
 * set_id, timing two evaluations after a warm-up with CUDA events on the
 * stream for each candidate, and keeps the fastest schedule for later
 * evaluations on this context (pepsi_get_schedule reads it), one field at a
 * time: the circuit chunk (the balanced chunk sizes of 32, 64, 128, ...,
 * 4096 layers for the set's mu, up to the one that holds every layer, stopping
 * at 4 GiB of chunk scratch or at the first that does not fit in memory),
 * then the threads per transform block (the default for N, half
 * and twice it), then for h = 4 and 8 the fused against the stored
 * relinearisation before the affine step, then the requests per shared
 * multiply-accumulate launch with its warp groups ((1), (2, 2), (2, 1),
 * (4, 2), (4, 1), timed on a batch of four copies of the request through
 * pepsi_eval_batch).  *chosen (may be NULL) receives
 * the chunk.  The result words do not depend on the schedule.
 * Synchronises the stream.  Errors: as pepsi_eval. */
int pepsi_autotune(pepsi_ctx* ctx, int set_id, const uint64_t* cts, void* stream, uint32_t* chosen);

/* Several requests in one call: request i is evaluated against server set
 * set_ids[i] exactly as by pepsi_eval (same output words), with mode
 * modes[i] (NULL: all indicator) and mask seed mask_seeds[i] (NULL: 0).
 * Requests on the same set are processed in groups of up to
 * pepsi_schedule.batch_requests (at most 4) whose
 * multiply-accumulate reads the server plaintexts once for the whole group
 * (or generates each plaintext chunk once, when the table is not
 * resident); the next group's multiply-accumulate overlaps the current
 * group's circuits on a second stream of the context.  cts[i]:
 * [B][ell][2][k][N], out_cts[i]: [B][2][r][N], each host or device.
 * Errors as pepsi_eval. */
int pepsi_eval_batch(pepsi_ctx* ctx, int nq, const int* set_ids, const uint64_t* const* cts, const int* modes,
                     const uint64_t* mask_seeds, uint64_t* const* out_cts, void* stream);

/* The same pipeline on layers [layer0, layer0+nl) only, returning the
 * per-layer intermediate words: h_out[B][nl][2][k][N] (h', coefficient form)
 * and e_out[B][nl][3][k][N] (the un-relinearised equality ciphertexts), host
 * or device; either may be NULL.  For sampled parity checks. */
int pepsi_eval_layers(pepsi_ctx* ctx, int set_id, const uint64_t* cts, uint32_t layer0, uint32_t nl,
                      uint64_t* h_out, uint64_t* e_out, void* stream);

/* Client result extraction (Algorithm 3): FV decryption, m = round(t z/Q)
 * mod t, slots of m.  ct: [2][k][N] (host or device); slots: host
 * uint32[N]; noise_budget_bits (may be NULL): log2(Q) - log2(2 max|[t z]_Q|).
 * Returns PEPSI_E_NOISE when the budget is not positive (slots are still
 * written). */
int pepsi_decrypt(pepsi_ctx* ctx, const uint64_t* ct, uint32_t* slots, double* noise_budget_bits);

/* The same over the first nprimes primes, modulus Q_r = q_0..q_{r-1}
 * (r = nprimes, 1..k): for a response switched by pepsi_mod_switch or
 * pepsi_params.response_primes.  ct: [2][r][N] (host or device); the budget
 * is log2(Q_r) - log2(2 max|[t z]_{Q_r}|).  Errors as pepsi_decrypt, and
 * PEPSI_E_PARAM for r outside 1..k. */
int pepsi_decrypt_primes(pepsi_ctx* ctx, const uint64_t* ct, uint32_t nprimes, uint32_t* slots,
                         double* noise_budget_bits);

/* Modulus switching of n ciphertexts to the first nprimes primes (the
 * server's response, whose size Section 7 reports as one ciphertext at one
 * prime): each coefficient's centred lift c~ in (-Q/2, Q/2] becomes
 * round(c~ q_0..q_{r-1} / Q) mod q_i, exact (Garner over the dropped
 * primes; Q / Q_r is odd, so there are no ties).  Decryption is preserved
 * while t (1 + |s|_1) / 2 plus the scaled noise stays below Q_r / 2.
 * ct: [n][2][k][N], out: [n][2][r][N], coefficient form, host or device;
 * r = k copies.  Errors: PEPSI_E_PARAM, PEPSI_E_CUDA. */
int pepsi_mod_switch(pepsi_ctx* ctx, const uint64_t* ct, size_t n, uint32_t nprimes, uint64_t* out, void* stream);

/* Forward (inverse = 0) or inverse negacyclic NTT over the ciphertext
 * primes, in place: polys[count][k][N], device memory.  Forward maps
 * coefficients to values at psi_i^(2 brev(j)+1) in position j. */
int pepsi_ntt(pepsi_ctx* ctx, uint64_t* polys, size_t count, int inverse, void* stream);

/* FV multiplication (Section 3.1) of n ciphertext pairs, exact textbook
 * rounding round(t/Q * a~ (x) b~): a, b [n][2][k][N], out [n][3][k][N]
 * (relin = 0) or [n][2][k][N] (relin = 1, RNS-digit relinearisation).
 * All coefficient form, device memory. */
int pepsi_ct_mult(pepsi_ctx* ctx, const uint64_t* a, const uint64_t* b, size_t n, int relin, uint64_t* out,
                  void* stream);

/* Relinearisation alone: in [n][3][k][N] -> out [n][2][k][N], coefficient
 * form, device memory. */
int pepsi_relin(pepsi_ctx* ctx, const uint64_t* in, size_t n, uint64_t* out, void* stream);

/* Size of the fixed device array used by pepsi_relin_noalloc. */
#define PEPSI_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Relinearisation that allocates nothing, for callers that cannot call
 * cudaMalloc: code running where another allocator has already reserved the
 * device memory (so cudaMalloc fails), and request loops that must not pay
 * for an allocation or for the device-wide synchronisation of cudaFree.
 * The paper has no counterpart; it is the same operation as pepsi_relin
 * (same arguments, same output words), with its scratch in a fixed device
 * array of PEPSI_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the
 * library holds until the process exits.
 * in: [n][3][k][N], out: [n][2][k][N], coefficient form, device memory.
 * The device the context was set up on must be the current device (its
 * launches go to the current device; another current device gives
 * PEPSI_E_PARAM).  The first call on a device looks up the array's device
 * address (once per device, with that device current); make that first
 * call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents, so calls that overlap on the GPU (other
 * streams, other threads, other contexts) race: serialise them.  Errors:
 * PEPSI_E_PARAM when n ciphertexts need more than the array holds
 * (((k+2) + 2) * k * N * 8 bytes each, so n at most
 * PEPSI_NOALLOC_SCRATCH_BYTES / that; pepsi_last_error gives the sizes),
 * when a buffer is not device memory, or when another device is current;
 * PEPSI_E_CUDA. */
int pepsi_relin_noalloc(pepsi_ctx* ctx, const uint64_t* in, size_t n, uint64_t* out, void* stream);

/* Test access to the keys: s (int8[N], host) and the relinearisation keys
 * in coefficient form rlk[k][2][k][N] (host); either may be NULL. */
int pepsi_export_keys(pepsi_ctx* ctx, int8_t* s, uint64_t* rlk);

/* Test of the bounded device waits (no counterpart in the paper): one
 * block waits on an mbarrier with the helper every multiply-accumulate
 * uses.  arrive = 1: the barrier completes and the call returns PEPSI_OK.
 * arrive = 0: nothing completes it, the wait gives up after about one
 * second, the kernel sets the context's error word and returns, and the
 * call returns PEPSI_E_TIMEOUT; the context stays usable (the error word
 * is cleared).  Synchronises the context's stream. */
int pepsi_wait_probe(pepsi_ctx* ctx, int arrive);

/* Measurement helper (no paper counterpart): the integer-pipe throughput of
 * the multiply forms the kernels use, measured on the current device with
 * 16 chains per thread on every SM, each step's multiplier taken from
 * another chain so that no product can be hoisted.  form = 1: 32x32->64
 * multiply-adds into 64-bit sums (mad.wide.u32, the multiply-accumulate's
 * inner operation); form = 2: the 32x32->64 product alone (mul.wide.u32);
 * form = 0: 32-bit multiply-adds (mad.lo.u32).  *ops_per_s receives
 * operations per second for the whole GPU.  Allocates 8 bytes of device
 * memory for the duration of the call. */
int pepsi_int_peak(int form, double* ops_per_s);

/* Per-kernel timing with CUDA events on the launching stream: enable (1) /
 * disable (0) and read back {launches, total milliseconds} per kernel
 * class (names[i] is a static string; returns the number of classes). */
int pepsi_profile_enable(pepsi_ctx* ctx, int on);
int pepsi_profile_read(pepsi_ctx* ctx, const char** names, uint64_t* launches, double* total_ms, int max);

/* ------------------------------------------------------------ engine
 * Continuous-batching request engine (no counterpart in the paper: the
 * served and batched forms of Algorithm 2's evaluation).  An engine serves
 * lanes; a lane is one (context, server set) pair with up to `slots`
 * requests in flight, evaluated by a carousel over the set's layers.  Each
 * step of a lane takes its next chunk of layers (the context's schedule
 * chunk; a chunk ends at the resident / regenerated boundary) and runs the
 * multiply-accumulate of that chunk for every request in the lane with one
 * read of the chunk's plaintexts (the kernel of pepsi_eval_batch), then
 * each request's equality circuits and layer sum.  A request admitted at a
 * step starts at the lane's current layer and is complete once it has
 * seen all mu layers, wrapping around.  The layer sum does not depend on
 * the order of the layers (with per-layer rounding, or with one rounding
 * for all layers), so every result has the words pepsi_eval gives.
 * Requests that arrive while others are on the GPU join at the lane's next
 * step, as slots and the HBM budget allow, and their work overlaps on the
 * device: each lane runs on streams of its own, and up to two steps per
 * lane are queued ahead of the GPU.  The per-request device state (the
 * request in NTT form, h' of a chunk, the layer sums) comes from a
 * stream-ordered memory pool of the engine; a request is admitted only
 * while the admitted requests' state fits hbm_budget. */
typedef struct pepsi_engine pepsi_engine;

typedef struct {
  pepsi_ctx* ctx;  /* the set's context; it must outlive the engine, and load no sets or
                      change its schedule or rounding while the engine exists */
  int set_id;      /* a set of ctx with one block of bins (bins = N) */
  uint32_t slots;  /* requests evaluated together, 1..4 */
} pepsi_lane;

typedef struct {
  uint64_t submitted, completed; /* requests */
  uint64_t steps;                /* lane steps enqueued */
  uint64_t bytes_in_use;         /* per-request device state of the admitted requests */
  uint64_t bytes_peak;           /* its maximum so far */
  uint64_t budget;               /* the admission budget in bytes */
} pepsi_engine_stats;

/* Create an engine over nlanes lanes.  Each lane gets a context of its own
 * that shares the lane context's keys, tables and sets (own streams and
 * scratch; the circuit scratch of one chunk per lane is allocated here).
 * hbm_budget: bytes of per-request state all admitted requests may hold
 * together (0: half of the free device memory after the lanes' scratch).
 * Errors: PEPSI_E_PARAM (a set with more than one block, slots outside
 * 1..4, a context whose rescale_group rounds runs of more than one layer
 * but fewer than all of them), PEPSI_E_NOMEM, PEPSI_E_CUDA. */
int pepsi_engine_create(const pepsi_lane* lanes, int nlanes, uint64_t hbm_budget, pepsi_engine** out);

/* Queue a request on a lane; thread-safe.  cts: [ell][2][k][N]
 * coefficient form, host (pinned memory keeps the copy asynchronous) or
 * device, read when the request is admitted; out_ct: [2][r][N] (r =
 * response_primes), host (pinned) or device, written when it completes.
 * Both must stay valid until pepsi_engine_wait reports the request done.
 * *ticket identifies it.  With client bins of gamma > 1 items, each of a
 * request's gamma batches is a request of its own: batch i with mask seed
 * mask_seed + i has the words of pepsi_eval's response i.  Errors:
 * PEPSI_E_PARAM (lane, mode, a value mode on a set without values, null
 * buffers). */
int pepsi_engine_submit(pepsi_engine* e, int lane, const uint64_t* cts, int mode, uint64_t mask_seed,
                        uint64_t* out_ct, uint64_t* ticket);

/* One scheduling pass by the calling thread: retire the steps the GPU has
 * completed, admit queued requests into free slots within the budget, and
 * queue each busy lane's next steps (at most two ahead).  Never waits for
 * the GPU.  *pending (may be NULL): requests submitted and not yet done.
 * A request whose admission or step fails is done with that error status
 * (pepsi_engine_wait returns it) and the others are still served; the call
 * returns the first such error of the pass.
 * Use either pepsi_engine_pump / pepsi_engine_run from one thread, or the
 * engine's own thread (pepsi_engine_start), not both. */
int pepsi_engine_pump(pepsi_engine* e, uint64_t* pending);

/* Pump until every request submitted so far is done; returns the first
 * failed request's status, else PEPSI_OK. */
int pepsi_engine_run(pepsi_engine* e);

/* Start / stop a thread of the engine that pumps continuously (it sleeps
 * about 20 microseconds between passes while work is in flight). */
int pepsi_engine_start(pepsi_engine* e);
int pepsi_engine_stop(pepsi_engine* e);

/* Wait until a request is done (pumping from the calling thread when no
 * engine thread runs); returns its status (PEPSI_OK, PEPSI_E_TIMEOUT when a
 * bounded device wait of its steps expired, PEPSI_E_NOMEM, PEPSI_E_CUDA).
 * latency_ms (may be NULL): from its submission to the engine seeing its
 * last step complete.  The engine forgets the ticket once this call has
 * reported it (tickets that are never waited for keep a few bytes each
 * until pepsi_engine_destroy).  Errors: PEPSI_E_PARAM for an unknown
 * ticket. */
int pepsi_engine_wait(pepsi_engine* e, uint64_t ticket, double* latency_ms);

/* Failure test of the engine (no counterpart in the paper): the next
 * admission on `lane` fails on the host with `status` (a PEPSI_E_* code)
 * instead of running, as if allocating or uploading the request had
 * failed.  That request is done with this status; the engine serves the
 * others.  Errors: PEPSI_E_PARAM. */
int pepsi_engine_fail_next(pepsi_engine* e, int lane, int status);

/* Counters of the engine. */
int pepsi_engine_get_stats(pepsi_engine* e, pepsi_engine_stats* out);

/* The batched form under a captured CUDA graph (no counterpart in the
 * paper).  Captures the evaluation of every request submitted and not yet
 * admitted into one graph: the engine schedules them exactly as
 * pepsi_engine_run would (slots and budget, lane steps), but queues the
 * whole schedule without waiting for the GPU, inside a stream capture
 * forked from `stream` (NULL: a stream of the graph) into every lane's
 * stream and joined back.  Nothing runs until pepsi_graph_launch; the
 * captured requests' tickets are done when this call returns.  Each launch
 * reads the same request buffers and writes the same output buffers again,
 * so refilling the request buffers and launching evaluates new requests of
 * the same shapes.  The requests must use device buffers; the engine's
 * thread must be stopped and no request may be in flight.  A launch must
 * not overlap another launch of a graph of the same engine or the engine's
 * own work (they share the lanes' scratch).  Errors: PEPSI_E_PARAM,
 * PEPSI_E_NOMEM, PEPSI_E_CUDA. */
typedef struct pepsi_graph pepsi_graph;
int pepsi_engine_capture(pepsi_engine* e, void* stream, pepsi_graph** out);

/* Launch a captured graph on `stream` (NULL: the graph's own stream).
 * synchronize = 1: wait for it and return PEPSI_E_TIMEOUT if a bounded
 * device wait of the evaluation expired. */
int pepsi_graph_launch(pepsi_graph* g, void* stream, int synchronize);

/* Wait for the graph's last launch and release it (NULL is ignored). */
void pepsi_graph_destroy(pepsi_graph* g);

/* Finish every request in flight, then release the engine and its lanes
 * (NULL is ignored). */
void pepsi_engine_destroy(pepsi_engine* e);

/* Release every device buffer of the context (NULL is ignored). */
void pepsi_destroy(pepsi_ctx* ctx);
/* Static description of an error code. */
const char* pepsi_strerror(int code);
/* Name and description of the last CUDA failure reported by a call of
 * this thread (valid until the next failing call). */
const char* pepsi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PEPSI_H */
