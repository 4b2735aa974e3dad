// Launch wrappers of the PEPSI kernels (host side).  All launches are
// asynchronous on the given stream; errors surface through
// cudaGetLastError() / the next synchronising call.
#pragma once
#include <cuda.h>

#include "common.cuh"

// Batched NTT over rows laid out [outer][np][N]: row r uses prime p0 + (r % np);
// src and dst may alias (in place).  fwd: coefficient -> evaluation form.
// split_out (forward only): dst receives the split operand format of the
// multiply-accumulate, and sums (rows laid out as dst's, 32-bit words) the
// sum of each word's two halves.
void launch_ntt(const DevView& V, bool fwd, const u64* src, u64* dst, size_t outer, int np, int p0, size_t src_os,
                size_t dst_os, cudaStream_t st, bool split_out = false, u32* sums = nullptr);

// A request prepared for the multiply-accumulate: its ell*2*k*N words in
// the split operand format, [ell][2][k][N], followed by the 32-bit sums of
// their halves in the same order (request_sums), 12 bytes per word in all.
inline size_t request_prepared_words(int ell, size_t kN) { return (size_t)ell * 3 * kN; }
inline u32* request_sums(u64* C, int ell, size_t kN) { return reinterpret_cast<u32*>(C + (size_t)ell * 2 * kN); }
inline const u32* request_sums(const u64* C, int ell, size_t kN) {
  return reinterpret_cast<const u32*>(C + (size_t)ell * 2 * kN);
}

// One round of the parallel cuckoo placement of m items into nbins bins of gamma
// slots (see pepsi_params.client_cuckoo): bins3[m][3] candidate bins; state[m]
// (1 = unplaced at the start), choice[m] (current candidate), claim[nbins]
// (all UINT32_MAX between rounds), slot_item[nbins][gamma] (-1 = free),
// load[nbins], evictions[nbins]; *unplaced (zeroed by the caller) receives the
// items left unplaced after the round.
void launch_cuckoo_round(const u32* bins3, u32 m, u32 nbins, u32 gamma, u32* claim, int32_t* slot_item, u32* load,
                         u32* evictions, uint8_t* state, uint8_t* choice, u32* unplaced, cudaStream_t st);

// CW-Encode of table entries (colex rank -> positions), pos[count][h], dummy -> PEPSI_CW_NONE.
void launch_cw_unrank(const u64* T, size_t count, const u64* binom, int ell, int h, uint16_t* pos, cudaStream_t st);

// Server plaintexts pt_s[l][j] in NTT form for L layers: P[L][ell][k][N], split operand format.
void launch_ptgen(const DevView& V, const uint16_t* pos, int L, int ell, int h, u64* P, cudaStream_t st);

// Plaintexts of L layers [L][ell][k][N]: either 64-bit words in the split
// operand format (w), or 7-byte words of the reduced values in three planes of
// the same shape (a: bits 0-31, b: bits 32-47, c: bits 48-55; every prime below
// 2^56).  Each base is 16-byte aligned.
struct PlainTab {
  const u64* w = nullptr;
  const u32* a = nullptr;
  const uint16_t* b = nullptr;
  const uint8_t* c = nullptr;
  bool packed() const { return a != nullptr; }
  // the table from word `off` on (a whole number of layers)
  PlainTab at(size_t off) const {
    PlainTab r;
    if (packed()) {
      r.a = a + off;
      r.b = b + off;
      r.c = c + off;
    } else {
      r.w = w + off;
    }
    return r;
  }
};
inline PlainTab plain_words(const u64* w) {
  PlainTab r;
  r.w = w;
  return r;
}

// Fused ct x pt multiply-accumulate: H[l][c][p][n] = sum_j C[j][c][p][n] * P[l][j][p][n] mod q_p.
// C a prepared request (split operand format and half sums), H reduced.  fold: terms between folds of the
// 64-bit partial sums.  *err is set when a bounded wait for a TMA copy expires.
// Returns cudaErrorInvalidValue when the tensor maps of the copies cannot be encoded.
cudaError_t launch_mac(const DevView& V, const u64* C, const PlainTab& P, u64* H, int ell, int L, int fold, int* err,
                       cudaStream_t st, int j0 = 0, int nj = -1, bool acc_in = false);

// The same for nq <= PEPSI_MAC_MAX_REQUESTS requests sharing the plaintexts: prepared request q
// at C[q], its h' [L][2][k][N] to H[q].  tile_points: 32
// or 64 points per block (16 or 8 layers); groups: 1 = each consumer thread serves every
// request, 2 = two groups of warps serve half of them each (2 or 4 requests; 3 requests
// always run in one group); one request runs launch_mac.
cudaError_t launch_mac_requests(const DevView& V, int nq, const u64* const* C, const PlainTab& P, u64* const* H,
                                int ell, int L, int fold, int* err, cudaStream_t st, int tile_points = 32,
                                int groups = 2);
// The same with the prepared requests back to back in C (request_prepared_words apart) and H[q]
// at H + q * hq.
cudaError_t launch_mac_multi(const DevView& V, const u64* C, int nq, const PlainTab& P, u64* H, size_t hq, int ell,
                             int L, int fold, int* err, cudaStream_t st, int tile_points = 32, int groups = 2);
// count split-format words (rows [..][k][N]) to the three planes of the 7-byte format, and back
// (reduced values)
void launch_pack7(const DevView& V, const u64* src, size_t count, u32* a, uint16_t* b, uint8_t* c, cudaStream_t st);
void launch_unpack7(const u32* a, const uint16_t* b, const uint8_t* c, size_t count, u64* out, cudaStream_t st);
constexpr int PEPSI_MAC_MAX_REQUESTS = 4;
// Per-request operands of the multi-request multiply-accumulate (passed by value).
struct MacRequests {
  CUtensorMap c[PEPSI_MAC_MAX_REQUESTS];  // request tiles
  CUtensorMap s[PEPSI_MAC_MAX_REQUESTS];  // their half sums
  u64* h[PEPSI_MAC_MAX_REQUESTS];         // h' outputs [L][2][k][N]
};

// In-place conversion of groups of k rows to (to = true) or from the split operand format.
void launch_split(const DevView& V, u64* x, size_t groups, bool to, cudaStream_t st);

// Exact centred base extension Q -> B of [L][2][k][N] coefficient rows into [L][2][kb][N].
// cst (k residues, may be NULL): also records side[l][j] = lift(x0 + cst) - lift(x0) mod p_j
// for coefficient 0 of component 0.
void launch_lift(const DevView& V, const u64* src, u64* dstB, int L, const u64* cst, u64* side, cudaStream_t st);

// Tensor product over Q u B of the NTT-form ciphertexts (A, B): (a0b0,
// a0b1+a1b0, a1b1), square: b = a; cstQ/side (may be NULL): constant added to
// component 0 of b (Q rows / B rows).  Each row is inverse-transformed in the
// same kernel: T3[L][3][k+kb][N] in coefficient form.
void launch_tensor_intt(const DevView& V, const u64* AQ, const u64* AB, const u64* BQ, const u64* BB,
                        const u64* cstQ, const u64* side, u64* T3, int L, bool square, cudaStream_t st);

// Exact round(t x / Q) from Q u B residues (coefficient form) -> D[L][3][k][N] mod Q.
// X[3][k+kb][N] (+)= sum over L layers of the tensor of (A, B) (NTT form over
// Q u B), each times the layer's value plaintext VP[l][k+kb][N] when VP is
// not null
void launch_tensor_sum(const DevView& V, const u64* AQ, const u64* AB, const u64* BQ, const u64* BB,
                       const u64* cstQ, const u64* side, const u64* VP, u64* X, int L, bool square, bool init,
                       cudaStream_t st);
// Constants of modulus switching from Q = q_0..q_{k-1} to Q_r = q_0..q_{r-1}
// (Q' = q_r..q_{k-1} dropped), computed on the host for each r.
struct ModSwitchArgs {
  int k = 0, r = 0;
  u64 h[PEPSI_MAXQ];                    // (Q' - 1)/2 mod q_p, every p
  u64 ginv[PEPSI_MAXQ][PEPSI_MAXQ];     // Garner over Q': d_l^-1 mod d_j (l < j), d_j = q_{r+j}
  u64 pw[PEPSI_MAXQ][PEPSI_MAXQ];       // prod_{l<j} d_l mod q_i, kept i
  u64 qdinv[PEPSI_MAXQ];                // Q'^-1 mod q_i, kept i
};
// bounded-wait test: *err = 1 after about one second unless arrive != 0
void launch_wait_probe(int arrive, int* err, cudaStream_t st);
// out[n][2][r][N] = round(c~ Q_r / Q) of in[n][2][k][N] (coefficient form)
void launch_modswitch(const DevView& V, const ModSwitchArgs& M, const u64* in, u64* out, size_t n, cudaStream_t st);
// Value plaintexts VP[L][k+kb][N] (NTT form) of the value rows vals[L][N]
void launch_valgen(const DevView& V, const u32* vals, int L, u64* VP, cudaStream_t st);
// acc[3][k][N] (+)= sum over L layers of D_l (NTT form over Q) times VP_l
void launch_accum_val(const DevView& V, const u64* D, const u64* VP, int L, u64* acc, bool init, cudaStream_t st);
void launch_scale_round(const DevView& V, const u64* T3, u64* D, int L, cudaStream_t st);

// RNS-digit relinearisation: D[L][3][k][N] coefficient form, rlk[k][2][k][N] NTT form
// -> R[L][2][k][N] NTT form.  DG: scratch [L][k+2][k][N].
void launch_relin(const DevView& V, const u64* D, const u64* rlk, u64* DG, u64* R, int L, cudaStream_t st);

// The digit transforms of launch_relin alone (DG[L][k+2][k][N]), and the key
// MAC fused with the affine step after it: out = R + z * H (rows [L][2][k][N],
// NTT form), stored, and its inverse NTT into coef, R never written.
void launch_relin_digits(const DevView& V, const u64* D, u64* DG, int L, cudaStream_t st);
void launch_relin_axpy_intt(const DevView& V, const u64* DG, const u64* rlk, const u64* zres, const u64* H, u64* out,
                            u64* coef, int L, cudaStream_t st);

// out = a + z * b over `groups` groups of k rows (z as k residues); out may alias a.
void launch_axpy(const DevView& V, const u64* a, const u64* zres, const u64* b, u64* out, size_t groups,
                 cudaStream_t st);

// The same, and the inverse NTT of out into coef (coefficient form) in one kernel; coef may alias b.
void launch_axpy_intt(const DevView& V, const u64* a, const u64* zres, const u64* b, u64* out, u64* coef,
                      size_t groups, cudaStream_t st);

// acc[3][k][N] (+)= sum_{l<L} D[l][3][k][N]
void launch_accum(const DevView& V, const u64* D, int L, u64* acc, bool init, cudaStream_t st);

// Client encryption of ell plaintexts given the client codeword positions pos[N][h].
void launch_encrypt(const DevView& V, const uint16_t* pos, int ell, int h, const u64* s_ntt, u64 seed, u64 idx0,
                    u64* cts, cudaStream_t st);

// Key generation: s (ternary) and its NTT rows; rlk in NTT form.
void launch_keygen(const DevView& V, u64 seed, int8_t* s, u64* s_ntt, u64* rlk, cudaStream_t st);

// Decryption: ct[2][k][N] -> slots[N] (u32) and max |[t z]_Q| as a double bit pattern in *maxr.
void launch_decrypt(const DevView& V, const u64* ct, const u64* s_ntt, u64* zbuf, u32* mbuf, u32* slots,
                    unsigned long long* maxr, cudaStream_t st);

// Cardinality mask: c0 += round(Q * Encode(r) / t), r uniform with sum 0 mod t.
void launch_mask(const DevView& V, u64 seed, u64* ct, cudaStream_t st);

// Configure kernels that need more than 48 KB of dynamic shared memory.
cudaError_t kernels_init(int N);

// Measured throughput (operations per second over the whole GPU) of
// 32x32->64 wide multiply-adds into 64-bit sums (form 1), wide products
// alone (form 2) or 32-bit multiply-adds (form 0).
double measure_int_peak(int form);
