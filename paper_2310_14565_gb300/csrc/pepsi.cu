// Context, orchestration and C ABI of the PEPSI GB300 library
// (declarations and contracts in include/pepsi.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "context.h"

using hostmath::u128;

namespace pepsi_detail {

thread_local std::string g_last_error = "no error";
thread_local std::string g_detail;

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PEPSI_OK;
  g_last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
  if (!g_detail.empty()) g_last_error += " (" + g_detail + ")";
  g_detail.clear();
  if (e == cudaErrorMemoryAllocation) return PEPSI_E_NOMEM;
  return PEPSI_E_CUDA;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaStream_t pick(pepsi_ctx* c, void* s) { return s ? (cudaStream_t)s : c->stream; }

// scratch slot `id` with at least `bytes`
void* scratch(pepsi_ctx* c, int id, size_t bytes, cudaError_t* err) {
  if ((int)c->scratch.size() <= id) c->scratch.resize(id + 1);
  DevBuf& b = c->scratch[id];
  if (b.bytes >= bytes && b.p) return b.p;
  if (b.p) {
    cudaStreamSynchronize(c->stream);
    cudaDeviceSynchronize();
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes ? bytes : 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = e;
    return nullptr;
  }
  b.bytes = bytes;
  return b.p;
}

// Free scratch slot `id` (after the device has finished with it).
void scratch_release(pepsi_ctx* c, int id) {
  if ((int)c->scratch.size() <= id || !c->scratch[id].p) return;
  cudaDeviceSynchronize();
  cudaFree(c->scratch[id].p);
  c->scratch[id].p = nullptr;
  c->scratch[id].bytes = 0;
}

void prof_collect(pepsi_ctx* c) {
  for (auto& pe : c->prof_ev) {
    float ms = 0;
    cudaEventSynchronize(pe.second.second);
    cudaEventElapsedTime(&ms, pe.second.first, pe.second.second);
    c->prof_ms[pe.first] += ms;
    c->ev_pool.push_back(pe.second.first);
    c->ev_pool.push_back(pe.second.second);
  }
  c->prof_ev.clear();
}

const u64* cst(pepsi_ctx* c, int slot) { return c->d_consts + (size_t)slot * c->k; }

// ------------------------------------------------------------ primitives
// NTT rows [outer][np][N] with prime offset p0.
void ntt(pepsi_ctx* c, bool fwd, const u64* src, u64* dst, size_t outer, int np, int p0, size_t sos, size_t dos,
         cudaStream_t st) {
  Prof p(c, PC_NTT, st);
  launch_ntt(c->V, fwd, src, dst, outer, np, p0, sos, dos, st);
}

// Arrays of the extension of L ciphertexts: Q part (NTT form, given) and
// B part (NTT form, computed).  src_ntt [L][2][k][N] -> coef (scratch) ->
// B [L][2][kb][N].  cstv: optional constant added to component 0 (side).
void extend(pepsi_ctx* c, const u64* src_ntt, u64* coef, u64* Bpart, int L, const u64* cstv, u64* side,
            cudaStream_t st) {
  const size_t kN = (size_t)c->k * c->N, kbN = (size_t)c->kb * c->N;
  ntt(c, false, src_ntt, coef, (size_t)L * 2, c->k, 0, kN, kN, st);
  {
    Prof p(c, PC_LIFT, st);
    launch_lift(c->V, coef, Bpart, L, cstv, side, st);
  }
  ntt(c, true, Bpart, Bpart, (size_t)L * 2, c->kb, c->k, kbN, kbN, st);
}

// relin(D) + z * H -> out, then extend(out): the key-switching sum and the
// affine step on the load of the inverse NTT (the relinearised product
// itself is not stored).
void relin_axpy_extend(pepsi_ctx* c, const u64* D, const u64* z, const u64* H, u64* out, u64* coef, u64* Bpart,
                       int L, const u64* cstv, u64* side, u64* Rtmp, cudaStream_t st);

// out = a + z * b, then extend(out) as above, the axpy on the load of the
// inverse NTT (coef may alias b).
void axpy_extend(pepsi_ctx* c, const u64* a, const u64* z, const u64* b, u64* out, u64* coef, u64* Bpart, int L,
                 const u64* cstv, u64* side, cudaStream_t st) {
  const size_t kbN = (size_t)c->kb * c->N;
  {
    Prof p(c, PC_NTT, st);
    launch_axpy_intt(c->V, a, z, b, out, coef, (size_t)L * 2, st);
  }
  {
    Prof p(c, PC_LIFT, st);
    launch_lift(c->V, coef, Bpart, L, cstv, side, st);
  }
  ntt(c, true, Bpart, Bpart, (size_t)L * 2, c->kb, c->k, kbN, kbN, st);
}

// T3 = tensor, then inverse NTT over Q u B, then exact scale-and-round -> D.
void mult_tail(pepsi_ctx* c, const u64* AQ, const u64* AB, const u64* BQ, const u64* BB, const u64* cQ,
               const u64* side, bool square, u64* T3, u64* D, int L, cudaStream_t st) {
  {
    Prof p(c, PC_TENSOR, st);  // the tensor and its inverse NTT over Q u B
    launch_tensor_intt(c->V, AQ, AB, BQ, BB, cQ, side, T3, L, square, st);
  }
  Prof p(c, PC_SCALE, st);
  launch_scale_round(c->V, T3, D, L, st);
}

// scratch id of the relinearisation digits (declared with the others below)
constexpr int kScratchDG = 40;
void relin(pepsi_ctx* c, const u64* D, u64* R, int L, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  u64* DG = (u64*)scratch(c, kScratchDG, (size_t)L * (c->k + 2) * c->k * c->N * 8, &e);
  if (!DG) return;  // the allocation error resurfaces through cudaGetLastError
  Prof p(c, PC_RELIN, st, 2);
  launch_relin(c->V, D, c->d_rlk, DG, R, L, st);
}

void relin_axpy_extend(pepsi_ctx* c, const u64* D, const u64* z, const u64* H, u64* out, u64* coef, u64* Bpart,
                       int L, const u64* cstv, u64* side, u64* Rtmp, cudaStream_t st) {
  if (!c->relin_fused) {  // the schedule's unfused form: R stored in Rtmp, then the affine step
    relin(c, D, Rtmp, L, st);
    axpy_extend(c, Rtmp, z, H, out, coef, Bpart, L, cstv, side, st);
    return;
  }
  const size_t kbN = (size_t)c->kb * c->N;
  cudaError_t e = cudaSuccess;
  u64* DG = (u64*)scratch(c, kScratchDG, (size_t)L * (c->k + 2) * c->k * c->N * 8, &e);
  if (!DG) return;  // the allocation error resurfaces through cudaGetLastError
  {
    Prof p(c, PC_RELIN, st, 2);
    launch_relin_digits(c->V, D, DG, L, st);
    launch_relin_axpy_intt(c->V, DG, c->d_rlk, z, H, out, coef, L, st);
  }
  {
    Prof p(c, PC_LIFT, st);
    launch_lift(c->V, coef, Bpart, L, cstv, side, st);
  }
  ntt(c, true, Bpart, Bpart, (size_t)L * 2, c->kb, c->k, kbN, kbN, st);
}


void axpy(pepsi_ctx* c, const u64* a, const u64* z, const u64* b, u64* out, size_t groups, cudaStream_t st) {
  Prof p(c, PC_POINTWISE, st);
  launch_axpy(c->V, a, z, b, out, groups, st);
}


cudaError_t eval_bufs(pepsi_ctx* c, int Lc, bool need_pc, EvalBufs* b) {
  cudaError_t e = cudaSuccess;
  const size_t N = c->N, k = c->k, kb = c->kb, np = k + kb;
  auto get = [&](int id, size_t words) { return (u64*)scratch(c, id, words * 8, &e); };
  b->C = get(S_C, request_prepared_words(c->ell, k * N));
  b->H = get(S_H, Lc * 2 * k * N);
  b->Hc = get(S_HC, Lc * 2 * k * N);
  b->XB = get(S_XB, Lc * 2 * kb * N);
  b->YB = get(S_YB, Lc * 2 * kb * N);
  b->T3 = get(S_T3, Lc * 3 * np * N);
  b->D = get(S_D, Lc * 3 * k * N);
  b->R = get(S_R, Lc * 2 * k * N);
  b->U = get(S_U, Lc * 2 * k * N);
  b->W = get(S_W, Lc * 2 * k * N);
  b->X = get(S_X, Lc * 2 * k * N);
  b->Y = get(S_Y, Lc * 2 * k * N);
  b->side = get(S_SIDE, Lc * kb + 1);
  b->acc = get(S_ACC, 3 * k * N);
  b->out = get(S_OUT, 3 * k * N);
  b->Pc = need_pc ? get(S_PC, (size_t)Lc * c->ell * k * N) : nullptr;
  if (e == cudaSuccess && (c->scratch.size() <= S_ZERO || !c->scratch[S_ZERO].p)) {
    b->zero = get(S_ZERO, 2 * k * N);
    if (b->zero) e = cudaMemset(b->zero, 0, 2 * k * N * 8);
  } else {
    b->zero = (u64*)c->scratch[S_ZERO].p;
  }
  return e;
}


// Arith-CW-Eq (Algorithm 1) on L layers whose h' is in H (NTT form), up to
// its last ciphertext product, whose operands are returned (h >= 2).  For
// h = 1 there is no product: D <- h' directly.  Hc <- h' in coefficient form.
LastMult eq_circuit_front(pepsi_ctx* c, EvalBufs& b, int L, cudaStream_t st) {
  const size_t k = c->k, N = c->N;
  const size_t ct2 = 2 * k * N;
  LastMult m;
  auto last = [&](const u64* AQ, const u64* AB, const u64* BQ, const u64* BB, const u64* cQ, const u64* side,
                  bool square) {
    m.AQ = AQ;
    m.AB = AB;
    m.BQ = BQ;
    m.BB = BB;
    m.cQ = cQ;
    m.side = side;
    m.square = square;
  };
  switch (c->h) {
    case 1: {
      ntt(c, false, b.H, b.Hc, (size_t)L * 2, c->k, 0, k * N, k * N, st);
      for (int l = 0; l < L; ++l) {
        cudaMemcpyAsync(b.D + (size_t)l * 3 * k * N, b.Hc + (size_t)l * ct2, ct2 * 8, cudaMemcpyDeviceToDevice, st);
        cudaMemsetAsync(b.D + (size_t)l * 3 * k * N + ct2, 0, k * N * 8, st);
      }
      break;
    }
    case 2: {  // E = Mult(h', h' - 1)
      extend(c, b.H, b.Hc, b.XB, L, cst(c, CS_D_TM1), b.side, st);
      last(b.H, b.XB, b.H, b.XB, cst(c, CS_D_TM1), b.side, false);
      break;
    }
    case 4: {  // u = R(h'^2) - 3h';  E = Mult(u, u + 2)
      extend(c, b.H, b.Hc, b.XB, L, nullptr, nullptr, st);
      mult_tail(c, b.H, b.XB, b.H, b.XB, nullptr, nullptr, true, b.T3, b.D, L, st);
      relin_axpy_extend(c, b.D, cst(c, CS_M3), b.H, b.U, b.X, b.YB, L, cst(c, CS_D_2), b.side, b.R, st);
      last(b.U, b.YB, b.U, b.YB, cst(c, CS_D_2), b.side, false);
      break;
    }
    case 8: {  // u = R(h'^2) - 7h'; w = R(u^2); E = Mult(w + 12u, w + 16u + 60)
      extend(c, b.H, b.Hc, b.XB, L, nullptr, nullptr, st);
      mult_tail(c, b.H, b.XB, b.H, b.XB, nullptr, nullptr, true, b.T3, b.D, L, st);
      relin_axpy_extend(c, b.D, cst(c, CS_M7), b.H, b.U, b.X, b.XB, L, nullptr, nullptr, b.R, st);
      mult_tail(c, b.U, b.XB, b.U, b.XB, nullptr, nullptr, true, b.T3, b.D, L, st);
      relin(c, b.D, b.W, L, st);
      axpy_extend(c, b.W, cst(c, CS_P12), b.U, b.X, b.R, b.XB, L, nullptr, nullptr, st);
      axpy_extend(c, b.W, cst(c, CS_P16), b.U, b.Y, b.U, b.YB, L, cst(c, CS_D_60), b.side, st);
      last(b.X, b.XB, b.Y, b.YB, cst(c, CS_D_60), b.side, false);
      break;
    }
  }
  return m;
}

// The whole circuit with per-layer rounding: D <- prod_{i<h}(h' - i) as
// un-relinearised 3-component ciphertexts (coefficient form).
void eq_circuit(pepsi_ctx* c, EvalBufs& b, int L, cudaStream_t st) {
  const LastMult m = eq_circuit_front(c, b, L, st);
  if (m.AQ) mult_tail(c, m.AQ, m.AB, m.BQ, m.BB, m.cQ, m.side, m.square, b.T3, b.D, L, st);
}


// Round the completed run in X into acc: inverse NTT over Q u B, exact
// round(t x / Q), accumulate (D serves as one layer of scratch).
void lazy_flush(pepsi_ctx* c, EvalBufs& b, LazyRun& r, cudaStream_t st) {
  const int np = c->k + c->kb;
  const size_t npN = (size_t)np * c->N;
  ntt(c, false, r.X, r.X, 3, np, 0, npN, npN, st);
  {
    Prof p(c, PC_SCALE, st);
    launch_scale_round(c->V, r.X, b.D, 1, st);
  }
  Prof p(c, PC_POINTWISE, st);
  launch_accum(c->V, b.D, 1, r.acc, r.acc_init, st);
  r.acc_init = false;
}

// Add the last products of the chunk's L layers to the run sums, rounding
// each run as it completes (and the final partial run when `end`).
// VP: value plaintexts of the chunk's layers [L][k+kb][N], or null.
void lazy_chunk(pepsi_ctx* c, EvalBufs& b, const LastMult& m, const u64* VP, int L, bool end, LazyRun& r,
                cudaStream_t st) {
  const size_t vstride = (size_t)(c->k + c->kb) * c->N;
  for (int done = 0; done < L;) {
    const u32 in_run = r.pos % r.G;
    const int take = (int)std::min<u32>((u32)(L - done), r.G - in_run);
    {
      const LastMult mm = m.at(c, done);
      Prof p(c, PC_TENSOR, st);
      launch_tensor_sum(c->V, mm.AQ, mm.AB, mm.BQ, mm.BB, mm.cQ, mm.side, VP ? VP + (size_t)done * vstride : nullptr,
                        r.X, take, mm.square, in_run == 0, st);
    }
    done += take;
    r.pos += take;
    if (r.pos % r.G == 0 || (end && done == L)) lazy_flush(c, b, r, st);
  }
}

// Run length of the lazy rescaling for an evaluation of nl layers in `mode`
// (1: per layer rounding; also for the value modes when B lacks the room).
u32 rescale_run(const pepsi_ctx* c, u32 nl, int mode) {
  const u32 g = c->prm.rescale_group;
  if (g <= 1 || c->h == 1) return 1;
  if (mode >= PEPSI_MODE_LABELS && !c->value_margin) return 1;
  return std::max<u32>(1, std::min<u32>(g == PEPSI_RESCALE_ALL ? nl : g, c->rescale_cap));
}

// Read and clear the device error flag (the stream must be synchronised).
bool take_error_flag(pepsi_ctx* c) {
  int v = 0;
  if (cudaMemcpy(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  if (v) cudaMemset(c->d_err, 0, sizeof(int));
  return v != 0;
}

// Name the failing step when a multiply-accumulate could not be launched.
cudaError_t mac_status(cudaError_t e) {
  if (e == cudaErrorInvalidValue)
    g_detail = "multiply-accumulate: the TMA tensor maps of the plaintext / request tiles could not be encoded";
  return e;
}

// Copy `bytes` between caller and device buffers through the stream.
cudaError_t copy_any(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
}

// a4: request ciphertexts (host or device) to NTT form, then to the split
// operand format of the multiply-accumulate with the sums of the halves,
// into C (request_prepared_words).
cudaError_t prepare_request(pepsi_ctx* c, const u64* cts, u64* C, cudaStream_t st) {
  const size_t kN = (size_t)c->k * c->N, words = (size_t)c->ell * 2 * kN;
  const u64* src = cts;
  if (!is_device_ptr(cts)) {
    CK(copy_any(C, cts, words * 8, st));
    src = C;
  }
  Prof p(c, PC_NTT, st);  // forward NTT, stored in the split operand format
  launch_ntt(c->V, true, src, C, (size_t)c->ell * 2, c->k, 0, kN, kN, st, true, request_sums(C, c->ell, kN));
  return cudaSuccess;
}

// Constants of modulus switching to the first r < k primes (host math):
// Garner over the dropped primes d_j = q_{r+j}, their prefix products and
// Q'^-1 mod the kept primes, (Q'-1)/2 mod every prime.
const ModSwitchArgs& ms_args(pepsi_ctx* c, int r) {
  if (!c->ms_args[r]) {
    auto M = std::make_unique<ModSwitchArgs>();
    M->k = c->k;
    M->r = r;
    const int m = c->k - r;
    for (int p = 0; p < c->k; ++p) {  // (Q'-1)/2 mod q_p: Q' is odd, so (Q'-1)/2 = (Q' - 1) * 2^-1
      const u64 q = c->Q[p];
      u64 qd = 1;
      for (int j = 0; j < m; ++j) qd = hostmath::mulmod(qd, c->Q[r + j] % q, q);
      M->h[p] = hostmath::mulmod((qd + q - 1) % q, (q + 1) / 2, q);
    }
    for (int j = 0; j < m; ++j)
      for (int l = 0; l < j; ++l) M->ginv[j][l] = hostmath::invmod(c->Q[r + l] % c->Q[r + j], c->Q[r + j]);
    for (int i = 0; i < r; ++i) {
      const u64 q = c->Q[i];
      u64 w = 1;
      for (int j = 0; j < m; ++j) {
        M->pw[i][j] = w;
        w = hostmath::mulmod(w, c->Q[r + j] % q, q);
      }
      M->qdinv[i] = hostmath::invmod(w, q);
    }
    c->ms_args[r] = std::move(M);
  }
  return *c->ms_args[r];
}

// RNS constants of the modulus Q_r = q_0..q_{r-1} (decryption over Q_r).
const RnsArgs& sub_args(pepsi_ctx* c, int r) {
  if (r == c->k) return c->rargs;
  if (!c->sub_args[r]) {
    auto A = std::make_unique<RnsArgs>(c->rargs);
    std::vector<u64> Qr(c->Q.begin(), c->Q.begin() + r);
    for (int j = 0; j < c->kb; ++j) A->pr[r + j] = c->rargs.pr[c->k + j];
    hostmath::rns_constants(Qr, c->B, c->t, &A->rc);
    A->k = r;
    c->sub_args[r] = std::move(A);
  }
  return *c->sub_args[r];
}

// a7 output: ct = (h!)^-1 * R(A) to coefficient form, plus the mask of
// Algorithm 5 in cardinality mode, switched to the response primes, copied
// to out (host or device).
cudaError_t finish_request(pepsi_ctx* c, EvalBufs& b, u64* acc, bool acc_ntt, int mode, u64 mask_seed, u64* out,
                           cudaStream_t st) {
  const size_t kN = (size_t)c->k * c->N;
  if (acc_ntt) ntt(c, false, acc, acc, 3, c->k, 0, kN, kN, st);  // value-weighted sum, NTT form
  relin(c, acc, b.R, 1, st);
  axpy(c, b.zero, cst(c, CS_ZINV), b.R, b.R, 2, st);
  ntt(c, false, b.R, b.out, 2, c->k, 0, kN, kN, st);
  if (mode == PEPSI_MODE_CARDINALITY || mode == PEPSI_MODE_SUM) {
    Prof p(c, PC_CLIENT, st);
    launch_mask(c->V, mask_seed, b.out, st);
  }
  if (c->resp < c->k) {  // response modulus switching (b.R is free after the relinearisation)
    {
      Prof p(c, PC_CLIENT, st);
      launch_modswitch(c->V, ms_args(c, c->resp), b.out, b.R, 1, st);
    }
    return copy_any(out, b.R, 2 * (size_t)c->resp * c->N * 8, st);
  }
  return copy_any(out, b.out, 2 * kN * 8, st);
}

// The copy stream of piecewise request uploads and its events, on first use.
cudaError_t ensure_copy_stream(pepsi_ctx* c) {
  if (c->copy_stream) return cudaSuccess;
  CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c->copy_ready, cudaEventDisableTiming));
  for (auto& ev : c->copy_ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  return cudaSuccess;
}

// scratch id of the lazy-rescaling run sum of a single request
constexpr int kScratchAccX = 46;
// scratch ids of the autotuner's response buffers
constexpr int kScratchTune = 48, kScratchTuneBatch = 49;
// scratch id of k zero residues (a zero scalar of the fused affine step)
constexpr int kScratchZeroK = 50;

// Core of pepsi_eval / pepsi_eval_layers.
int eval_core(pepsi_ctx* c, int set_id, const u64* cts, u32 layer0, u32 nl, int mode, u64 mask_seed, u64* out_ct,
              u64* h_out, u64* e_out, cudaStream_t st) {
  if (set_id < 0 || set_id >= (int)c->sets.size() || !c->sets[set_id].live) return PEPSI_E_PARAM;
  ServerSet& S = c->sets[set_id];
  if ((u64)layer0 + nl > S.mu || !cts) return PEPSI_E_PARAM;
  if (mode < PEPSI_MODE_INDICATOR || mode > PEPSI_MODE_SUM) return PEPSI_E_PARAM;
  const bool valued = mode >= PEPSI_MODE_LABELS;
  if (valued && !S.has_values) return PEPSI_E_PARAM;
  const size_t k = c->k, N = c->N;
  const size_t vstride = (size_t)(c->k + c->kb) * N;  // value plaintext words per layer
  const size_t kN = k * N, ct2 = 2 * kN, ct3 = 3 * kN;
  const int Lc = balanced_chunk(c->chunk, nl);
  const u32 end = layer0 + nl, res_end = std::min(end, S.mu_res);
  EvalBufs b;
  cudaError_t e = eval_bufs(c, Lc, res_end < end, &b);
  if (e != cudaSuccess) return cuda_status(e);
  // per-layer E words are only defined with per-layer rounding
  const u32 G = e_out ? 1 : rescale_run(c, nl, mode);
  LazyRun lr{};
  if (G > 1) {
    lr.X = (u64*)scratch(c, kScratchAccX, (size_t)3 * (c->k + c->kb) * N * 8, &e);
    if (!lr.X) return cuda_status(e);
    lr.acc = b.acc;
    lr.G = G;
  }
  // A host request with resident layers arrives in pieces of its code bits:
  // the upload of piece p+1 overlaps the NTT and multiply-accumulate of
  // piece p, each piece's MAC adding into h' (the MAC is a sum over the
  // bits).  Otherwise the request is prepared whole.
  constexpr int npieces = pepsi_ctx::kPieces;
  const bool pieces = !is_device_ptr(cts) && res_end > layer0 && c->ell >= 4 * npieces;
  if (!pieces) CKS(prepare_request(c, cts, b.C, st));
  // a5 on the resident layers: a multiply-accumulate launch over all of
  // them (one per piece), so the request is read from HBM once
  u64* Hall = nullptr;
  if (res_end > layer0) {
    Hall = (u64*)scratch(c, S_HALL, (size_t)(res_end - layer0) * ct2 * 8, &e);
    if (!Hall) return cuda_status(e);
    const PlainTab P0 = S.plain(kN, c->ell, layer0);
    if (pieces) {
      // Piece boundaries in multiples of 4 bits.  The first piece is short, so
      // that little of the upload is exposed, yet its NTT and MAC must cover
      // the upload of the rest.  The MAC reads nres*ell*k*N table words while
      // the rest of the request is 2*(ell - j1)*k*N words, copied from the host
      // at well over 1/32 of HBM bandwidth: j1 = 64/nres of the bits covers it,
      // at least 4 bits and at most half.
      static_assert(pepsi_ctx::kPieces == 2, "two pieces");
      const double w = std::min(0.5, 64.0 / (double)(res_end - layer0));
      const int j1 = std::max(4, std::min((int)(c->ell * w) & ~3, (c->ell / 2) & ~3));
      const int jb[3] = {0, j1, c->ell};
      CKS(ensure_copy_stream(c));
      CKS(cudaEventRecord(c->copy_ready, st));  // earlier work on st no longer reads the request buffer
      CKS(cudaStreamWaitEvent(c->copy_stream, c->copy_ready, 0));
      for (int q = 0; q < npieces; ++q) {
        CKS(cudaMemcpyAsync(b.C + (size_t)jb[q] * ct2, cts + (size_t)jb[q] * ct2,
                            (size_t)(jb[q + 1] - jb[q]) * ct2 * 8, cudaMemcpyHostToDevice, c->copy_stream));
        CKS(cudaEventRecord(c->copy_ev[q], c->copy_stream));
      }
      for (int q = 0; q < npieces; ++q) {
        CKS(cudaStreamWaitEvent(st, c->copy_ev[q], 0));
        {
          Prof p(c, PC_NTT, st);  // forward NTT of the piece, stored in the split format
          launch_ntt(c->V, true, b.C + (size_t)jb[q] * ct2, b.C + (size_t)jb[q] * ct2,
                     (size_t)(jb[q + 1] - jb[q]) * 2, c->k, 0, kN, kN, st, true,
                     request_sums(b.C, c->ell, kN) + (size_t)jb[q] * ct2);
        }
        Prof p(c, PC_MAC, st);
        CKS(mac_status(launch_mac(c->V, b.C, P0, Hall, c->ell, (int)(res_end - layer0), c->mac_fold, c->d_err, st,
                                  jb[q], jb[q + 1] - jb[q], q > 0)));
      }
    } else {
      Prof p(c, PC_MAC, st);
      CKS(mac_status(launch_mac(c->V, b.C, P0, Hall, c->ell, (int)(res_end - layer0), c->mac_fold, c->d_err, st)));
    }
  }
  bool first = true;
  u64* const Hchunk = b.H;  // h' of a regenerated chunk (Lc layers)
  for (u32 l0 = layer0; l0 < end;) {
    int L = (int)std::min<u32>(Lc, end - l0);
    if (l0 < res_end) {
      L = (int)std::min<u32>(L, res_end - l0);
      b.H = Hall + (size_t)(l0 - layer0) * ct2;
    } else {
      b.H = Hchunk;
      {
        Prof p(c, PC_PTGEN, st);
        launch_ptgen(c->V, S.dpos + (size_t)l0 * N * c->h, L, c->ell, c->h, b.Pc, st);
      }
      Prof p(c, PC_MAC, st);  // a5 on a regenerated chunk
      CKS(mac_status(launch_mac(c->V, b.C, plain_words(b.Pc), b.H, c->ell, L, c->mac_fold, c->d_err, st)));
    }
    const u64* VP = valued ? S.dVP + (size_t)l0 * vstride : nullptr;
    if (G > 1) {  // a6 + a7 with lazy rescaling
      const LastMult m = eq_circuit_front(c, b, L, st);
      lazy_chunk(c, b, m, VP, L, l0 + L == end, lr, st);
    } else {
      eq_circuit(c, b, L, st);  // a6
      if (e_out) CKS(copy_any(e_out + (size_t)(l0 - layer0) * ct3, b.D, (size_t)L * ct3 * 8, st));
      if (valued) {  // a7, Algorithms 4-5: sum of val_s[i'] * E_{i'} in NTT form
        ntt(c, true, b.D, b.D, (size_t)L * 3, c->k, 0, k * N, k * N, st);
        Prof p(c, PC_POINTWISE, st);
        launch_accum_val(c->V, b.D, VP, L, b.acc, first, st);
      } else {
        Prof p(c, PC_POINTWISE, st);  // a7: layer accumulation
        launch_accum(c->V, b.D, L, b.acc, first, st);
      }
    }
    // b.Hc holds h' in coefficient form after the circuit
    if (h_out) CKS(copy_any(h_out + (size_t)(l0 - layer0) * ct2, b.Hc, (size_t)L * ct2 * 8, st));
    first = false;
    l0 += L;
  }
  if (out_ct) CKS(finish_request(c, b, b.acc, valued && G == 1, mode, mask_seed, out_ct, st));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  if (!is_device_ptr(out_ct ? (const void*)out_ct : (const void*)b.out) || (h_out && !is_device_ptr(h_out)) ||
      (e_out && !is_device_ptr(e_out))) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (take_error_flag(c)) return PEPSI_E_TIMEOUT;
  }
  if (c->prof) prof_collect(c);
  return PEPSI_OK;
}

// Core of pepsi_eval_batch: requests grouped by server set, up to
// batch_requests (at most PEPSI_MAC_MAX_REQUESTS) per group; each group's multiply-accumulate reads
// the plaintexts once (resident table) or generates each chunk once
// (streamed table); the equality circuits then run request by request.
// With a resident table the multiply-accumulate of the next group runs on
// the context's second stream while the circuits of the current group run
// on the call's stream (double-buffered requests and h'), so the
// HBM-bound stream of plaintexts overlaps the compute-bound circuits.
enum { S_CB = 41, S_HB = 42, S_ACCB = 43, S_CB2 = 44, S_HB2 = 45, S_ACCXB = 47 };
int eval_batch_core(pepsi_ctx* c, int nq, const int* set_ids, const u64* const* cts, const int* modes,
                    const u64* mask_seeds, u64* const* outs, cudaStream_t st) {
  const size_t k = c->k, N = c->N, kN = k * N, ct2 = 2 * kN, ct3 = 3 * kN;
  const size_t cwords = request_prepared_words(c->ell, kN);
  for (int i = 0; i < nq; ++i) {
    if (set_ids[i] < 0 || set_ids[i] >= (int)c->sets.size() || !c->sets[set_ids[i]].live || !cts[i] || !outs[i])
      return PEPSI_E_PARAM;
    const int mode = modes ? modes[i] : PEPSI_MODE_INDICATOR;
    if (mode < PEPSI_MODE_INDICATOR || mode > PEPSI_MODE_SUM) return PEPSI_E_PARAM;
    if (mode >= PEPSI_MODE_LABELS && !c->sets[set_ids[i]].has_values) return PEPSI_E_PARAM;
  }
  // groups of requests on the same set, in order of first appearance
  std::vector<std::vector<int>> groups;
  {
    std::vector<char> done(nq, 0);
    for (int i0 = 0; i0 < nq; ++i0) {
      if (done[i0]) continue;
      std::vector<int> grp;
      for (int i = i0; i < nq && (int)grp.size() < c->batch_requests; ++i)
        if (!done[i] && set_ids[i] == set_ids[i0]) grp.push_back(i);
      for (int i : grp) done[i] = 1;
      groups.push_back(grp);
    }
  }
  cudaError_t e = cudaSuccess;
  if (!c->aux_stream) {
    CKS(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 4; ++i) CKS(cudaEventCreateWithFlags(&c->aux_ev[i], cudaEventDisableTiming));
  }
  cudaStream_t ax = c->aux_stream;
  cudaEvent_t mac_done[2] = {c->aux_ev[0], c->aux_ev[1]}, circ_done[2] = {c->aux_ev[2], c->aux_ev[3]};
  // the auxiliary stream starts after everything already queued on the call's stream
  CKS(cudaEventRecord(circ_done[0], st));
  CKS(cudaEventRecord(circ_done[1], st));
  bool any_host = false;
  int slot = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::vector<int>& grp = groups[gi];
    const int G = (int)grp.size();
    ServerSet& S = c->sets[set_ids[grp[0]]];
    const u32 mu = S.mu, mres = S.mu_res;
    const int Lc = balanced_chunk(c->chunk, mu);
    EvalBufs b;
    e = eval_bufs(c, Lc, mres < mu, &b);
    if (e != cudaSuccess) return cuda_status(e);
    const size_t hq = (size_t)std::max<u32>(mres, (u32)Lc) * ct2;
    u64* CB = (u64*)scratch(c, slot ? S_CB2 : S_CB, (size_t)PEPSI_MAC_MAX_REQUESTS * cwords * 8, &e);
    u64* HB = (u64*)scratch(c, slot ? S_HB2 : S_HB, (size_t)PEPSI_MAC_MAX_REQUESTS * hq * 8, &e);
    u64* ACC = (u64*)scratch(c, S_ACCB, (size_t)PEPSI_MAC_MAX_REQUESTS * ct3 * 8, &e);
    if (!CB || !HB || !ACC) return cuda_status(e);
    // per request: its mode, value plaintexts and rounding run length
    const size_t xw = (size_t)3 * (c->k + c->kb) * N, vstride = (size_t)(c->k + c->kb) * N;
    int gmode[PEPSI_MAC_MAX_REQUESTS];
    LazyRun lr[PEPSI_MAC_MAX_REQUESTS];
    u64* ACCX = nullptr;
    for (int g = 0; g < G; ++g) {
      gmode[g] = modes ? modes[grp[g]] : PEPSI_MODE_INDICATOR;
      lr[g].G = rescale_run(c, mu, gmode[g]);
      lr[g].acc = ACC + (size_t)g * ct3;
      if (lr[g].G > 1) {
        if (!ACCX) ACCX = (u64*)scratch(c, S_ACCXB, (size_t)PEPSI_MAC_MAX_REQUESTS * xw * 8, &e);
        if (!ACCX) return cuda_status(e);
        lr[g].X = ACCX + (size_t)g * xw;
      }
    }
    if (mres) {
      // requests and multiply-accumulate over the resident layers on the auxiliary
      // stream, once the circuits that last used this slot's buffers are done
      CKS(cudaStreamWaitEvent(ax, circ_done[slot], 0));
      for (int g = 0; g < G; ++g) CKS(prepare_request(c, cts[grp[g]], CB + (size_t)g * cwords, ax));
      {
        Prof p(c, PC_MAC, ax);
        CKS(mac_status(launch_mac_multi(c->V, CB, G, S.plain(kN, c->ell), HB, hq, c->ell, (int)mres, c->mac_fold,
                                        c->d_err, ax, c->batch_points, c->batch_groups)));
      }
      CKS(cudaEventRecord(mac_done[slot], ax));
      CKS(cudaStreamWaitEvent(st, mac_done[slot], 0));
    } else {
      for (int g = 0; g < G; ++g) CKS(prepare_request(c, cts[grp[g]], CB + (size_t)g * cwords, st));
    }
    for (u32 l0 = 0; l0 < mu;) {
      int L = (int)std::min<u32>(Lc, mu - l0);
      const bool res = l0 < mres;
      if (res) {
        L = (int)std::min<u32>(L, mres - l0);
      } else {
        {
          Prof p(c, PC_PTGEN, st);
          launch_ptgen(c->V, S.dpos + (size_t)l0 * N * c->h, L, c->ell, c->h, b.Pc, st);
        }
        Prof p(c, PC_MAC, st);
        CKS(mac_status(launch_mac_multi(c->V, CB, G, plain_words(b.Pc), HB, hq, c->ell, L, c->mac_fold, c->d_err, st,
                                        c->batch_points, c->batch_groups)));
      }
      for (int g = 0; g < G; ++g) {
        b.H = HB + (size_t)g * hq + (res ? (size_t)l0 * ct2 : 0);
        const u64* VP = gmode[g] >= PEPSI_MODE_LABELS ? S.dVP + (size_t)l0 * vstride : nullptr;
        if (lr[g].G > 1) {
          const LastMult m = eq_circuit_front(c, b, L, st);
          lazy_chunk(c, b, m, VP, L, l0 + L == mu, lr[g], st);
          continue;
        }
        eq_circuit(c, b, L, st);
        if (VP) {
          ntt(c, true, b.D, b.D, (size_t)L * 3, c->k, 0, kN, kN, st);
          Prof p(c, PC_POINTWISE, st);
          launch_accum_val(c->V, b.D, VP, L, ACC + (size_t)g * ct3, l0 == 0, st);
        } else {
          Prof p(c, PC_POINTWISE, st);
          launch_accum(c->V, b.D, L, ACC + (size_t)g * ct3, l0 == 0, st);
        }
      }
      l0 += L;
    }
    for (int g = 0; g < G; ++g) {
      const int i = grp[g];
      CKS(finish_request(c, b, ACC + (size_t)g * ct3, gmode[g] >= PEPSI_MODE_LABELS && lr[g].G == 1, gmode[g],
                         mask_seeds ? mask_seeds[i] : 0, outs[i], st));
      any_host |= !is_device_ptr(outs[i]);
    }
    CKS(cudaEventRecord(circ_done[slot], st));
    slot ^= 1;
  }
  // nothing may remain queued on the auxiliary stream after the call's stream completes
  CKS(cudaEventRecord(mac_done[0], ax));
  CKS(cudaStreamWaitEvent(st, mac_done[0], 0));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  if (any_host) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (take_error_flag(c)) return PEPSI_E_TIMEOUT;
  }
  if (c->prof) prof_collect(c);
  return PEPSI_OK;
}

int validate(const pepsi_params* p) {
  if (!p) return PEPSI_E_PARAM;
  if (p->N < 16 || p->N > 16384 || (p->N & (p->N - 1))) return PEPSI_E_PARAM;
  if (p->k < 1 || p->k > PEPSI_MAXQ) return PEPSI_E_PARAM;
  for (u32 i = 0; i < p->k; ++i)
    if (p->prime_bits[i] < 20 || p->prime_bits[i] > 60) return PEPSI_E_PARAM;
  if (p->t < 3 || p->t >= (1ull << 32) || (p->t - 1) % (2ull * p->N) || !hostmath::is_prime(p->t))
    return PEPSI_E_PARAM;
  if (p->h != 1 && p->h != 2 && p->h != 4 && p->h != 8) return PEPSI_E_PARAM;
  if (p->num_hashes != 3 && p->num_hashes != 0) return PEPSI_E_PARAM;
  u32 logb = 0;
  while ((1u << logb) < p->N) ++logb;
  if (p->lambda_bar < 1 || p->lambda_bar + logb >= 64) return PEPSI_E_PARAM;
  return PEPSI_OK;
}

cudaError_t upload(void** dst, const void* src, size_t bytes) {
  CK(cudaMalloc(dst, bytes));
  return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
}

void free_set(ServerSet& S) {
  cudaFree(S.dT);
  cudaFree(S.dpos);
  cudaFree(S.dP);
  cudaFree(S.dVP);
  S = ServerSet{};
}

pepsi_ctx* ctx_fork(const pepsi_ctx* p, cudaError_t* err) {
  pepsi_ctx* c = new pepsi_ctx();
  c->borrowed = true;
  c->prm = p->prm;
  c->device = p->device;
  c->N = p->N;
  c->logN = p->logN;
  c->k = p->k;
  c->kb = p->kb;
  c->ell = p->ell;
  c->h = p->h;
  c->t = p->t;
  c->Q = p->Q;
  c->B = p->B;
  c->psi = p->psi;
  c->psi_t = p->psi_t;
  c->log2q = p->log2q;
  c->rargs = p->rargs;
  c->V = p->V;
  c->V.host_args = &c->rargs;
  c->d_pr = p->d_pr;
  c->d_twp = p->d_twp;
  c->d_itwp = p->d_itwp;
  c->d_rc = p->d_rc;
  c->d_binom = p->d_binom;
  c->d_s = p->d_s;
  c->d_s_ntt = p->d_s_ntt;
  c->d_rlk = p->d_rlk;
  c->d_consts = p->d_consts;
  c->mac_fold = p->mac_fold;
  for (const ServerSet& S : p->sets) {  // device views only; the host tables stay with the parent
    ServerSet F;
    F.live = S.live;
    F.mu = S.mu;
    F.dT = S.dT;
    F.dpos = S.dpos;
    F.dP = S.dP;
    F.p7 = S.p7;
    F.mu_res = S.mu_res;
    F.has_values = S.has_values;
    F.dVP = S.dVP;
    c->sets.push_back(std::move(F));
  }
  for (const SetGroup& G : p->groups) {
    SetGroup F;
    F.live = G.live;
    F.mu = G.mu;
    F.blk = G.blk;
    F.has_values = G.has_values;
    c->groups.push_back(std::move(F));
  }
  c->logb = p->logb;
  c->blocks = p->blocks;
  c->gamma = p->gamma;
  c->chunk = p->chunk;
  c->relin_fused = p->relin_fused;
  c->batch_points = p->batch_points;
  c->batch_groups = p->batch_groups;
  c->batch_requests = p->batch_requests;
  c->rescale_cap = p->rescale_cap;
  c->value_margin = p->value_margin;
  c->resp = p->resp;
  c->p7 = p->p7;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = e;
    pepsi_destroy(c);
    return nullptr;
  }
  return c;
}

}  // namespace pepsi_detail

using namespace pepsi_detail;

// ====================================================== no-allocation path
// Relinearisation whose scratch lives in a fixed device array instead of
// memory from cudaMalloc, for callers that cannot allocate (see
// pepsi_relin_noalloc in pepsi.h).  The array is part of this module: every
// device that loads the library holds PEPSI_NOALLOC_SCRATCH_BYTES of it
// until the process exits, and all calls share it.
static __device__ __align__(256) u64 g_noalloc_scratch[PEPSI_NOALLOC_SCRATCH_BYTES / sizeof(u64)];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
u64* g_noalloc_addr[kMaxDevices] = {};

// Device address of the array on the context's device.  In host code the
// array's name only stands for it; cudaGetSymbolAddress gives the address
// that kernels may use.  Looked up once per device, with that device
// current: the context's device must be the current one (every launch of
// the call goes to the current device), else PEPSI_E_PARAM.
int noalloc_scratch(const pepsi_ctx* c, u64** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev != c->device) {
    g_last_error = "pepsi_relin_noalloc: the context was set up on device " + std::to_string(c->device) +
                   " but device " + std::to_string(dev) + " is current";
    return PEPSI_E_PARAM;
  }
  if (dev < 0 || dev >= kMaxDevices) return PEPSI_E_PARAM;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e);
    g_noalloc_addr[dev] = static_cast<u64*>(p);
  }
  *out = g_noalloc_addr[dev];
  return PEPSI_OK;
}
}  // namespace

// ================================================================ C ABI
extern "C" {

const char* pepsi_last_error(void) { return g_last_error.c_str(); }

const char* pepsi_strerror(int code) {
  switch (code) {
    case PEPSI_OK: return "ok";
    case PEPSI_E_PARAM: return "invalid or unsupported parameters";
    case PEPSI_E_BIN_OVERFLOW: return "server bin overflow (more than mu items in a bin)";
    case PEPSI_E_CUCKOO_FAIL: return "cuckoo hashing failed (eviction bound reached)";
    case PEPSI_E_NOMEM: return "device memory exhausted";
    case PEPSI_E_CUDA: return "CUDA runtime error";
    case PEPSI_E_TIMEOUT: return "bounded device wait expired";
    case PEPSI_E_NOISE: return "noise budget exhausted";
    default: return "unknown error";
  }
}

void pepsi_destroy(pepsi_ctx* c) {
  if (!c) return;
  if (c->borrowed) {  // a lane: only its own streams, events, error word and scratch
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->aux_stream) cudaStreamSynchronize(c->aux_stream);
    for (auto& b : c->scratch) cudaFree(b.p);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto& pe : c->prof_ev) {
      cudaEventDestroy(pe.second.first);
      cudaEventDestroy(pe.second.second);
    }
    cudaFree(c->d_err);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->copy_ready) cudaEventDestroy(c->copy_ready);
    for (auto ev : c->copy_ev)
      if (ev) cudaEventDestroy(ev);
    for (auto ev : c->aux_ev)
      if (ev) cudaEventDestroy(ev);
    delete c;
    return;
  }
  cudaDeviceSynchronize();
  for (auto& S : c->sets) free_set(S);
  for (auto& b : c->scratch) cudaFree(b.p);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (auto& pe : c->prof_ev) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  cudaFree(c->d_pr);
  cudaFree(c->d_twp);
  cudaFree(c->d_itwp);
  cudaFree(c->d_rc);
  cudaFree(c->d_binom);
  cudaFree(c->d_s);
  cudaFree(c->d_s_ntt);
  cudaFree(c->d_rlk);
  cudaFree(c->d_consts);
  cudaFree(c->d_err);
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->copy_ready) cudaEventDestroy(c->copy_ready);
  for (auto ev : c->copy_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto ev : c->aux_ev)
    if (ev) cudaEventDestroy(ev);
  delete c;
}

int pepsi_setup(const pepsi_params* params, uint64_t key_seed, pepsi_ctx** out) {
  if (!out) return PEPSI_E_PARAM;
  *out = nullptr;
  int rc = validate(params);
  if (rc) return rc;
  pepsi_ctx* c = new pepsi_ctx();
  c->prm = *params;
  c->N = (int)params->N;
  while ((1 << c->logN) < c->N) ++c->logN;
  c->k = (int)params->k;
  c->t = params->t;
  c->h = (int)params->h;
  c->ell = params->ell ? (int)params->ell : (int)hostmath::code_length(params->lambda_bar, params->h);
  if (c->ell <= 0 || c->ell > 65535 || hostmath::binom_sat(c->ell, c->h) < (1ull << params->lambda_bar)) {
    delete c;
    return PEPSI_E_PARAM;
  }
  if (const char* ch = getenv("PEPSI_CHUNK")) c->chunk = std::max(1, atoi(ch));
  // primes
  for (int i = 0; i < c->k; ++i) {
    u64 q = hostmath::find_prime(params->prime_bits[i], c->N, c->Q);
    if (!q) {
      delete c;
      return PEPSI_E_PARAM;
    }
    c->Q.push_back(q);
  }
  double lq = 0;
  for (u64 q : c->Q) lq += std::log2((double)q);
  c->log2q = lq;
  // lazy sums in the MAC must stay below 2^128
  {
    u64 qmax = *std::max_element(c->Q.begin(), c->Q.end());
    long double bound = (long double)c->ell * (long double)(qmax - 1) * (long double)(qmax - 1);
    if (bound >= std::ldexp(1.0L, 127)) {
      delete c;
      return PEPSI_E_PARAM;
    }
  }
  {  // bins: B blocks of N slots
    const u64 bins = params->bins ? params->bins : (u64)c->N;
    if (bins < (u64)c->N || bins % c->N || (bins & (bins - 1)) || bins / c->N > 1024) {
      delete c;
      return PEPSI_E_PARAM;
    }
    while ((1ull << c->logb) < bins) ++c->logb;
    c->blocks = (u32)(bins / c->N);
    if (params->lambda_bar + c->logb >= 64) {
      delete c;
      return PEPSI_E_PARAM;
    }
  }
  if (params->response_primes > (u32)c->k || params->gamma > 16 || params->client_cuckoo > 1) {
    delete c;
    return PEPSI_E_PARAM;
  }
  c->gamma = params->gamma ? params->gamma : 1;
  c->resp = params->response_primes ? (int)params->response_primes : c->k;
  // resident plaintexts in 7 bytes per word on request (every q_i < 2^56)
  {
    bool fits = true;
    for (u64 q : c->Q) fits = fits && q < (1ull << 56);
    const u32 pb = params->plaintext_bytes;
    if ((pb != 0 && pb != 7 && pb != 8) || (pb == 7 && !fits)) {
      delete c;
      return PEPSI_E_PARAM;
    }
    c->p7 = pb == 7;
  }
  // lazy rescaling: runs of up to rescale_cap layers share one rounding
  {
    const u32 g = params->rescale_group;
    c->rescale_cap = g <= 1 ? 1 : g != PEPSI_RESCALE_ALL ? g : params->mu ? params->mu : 65536u;
  }
  // auxiliary base B: primes with log2 B >= log2(t N Q G) + 3, G the
  // longest run of layers whose exact products are summed before rounding
  // (and, for the value modes, N t / 2 times more: the product with a value
  // plaintext of centred coefficients).  59-bit primes where as few of them
  // cover the bound as of 61-bit ones (their forward transforms then skip the
  // per-stage reduction: 32 q < 2^64), else 61-bit primes.
  c->value_margin = params->server_values != 0 && c->rescale_cap > 1;
  const double needB = std::log2((double)c->t) + c->logN + lq + std::ceil(std::log2((double)c->rescale_cap)) + 3.0 +
                       (c->value_margin ? std::ceil(c->logN + std::log2((double)c->t) - 1.0) : 0.0);
  const int bbits = std::ceil(needB / 58.9) <= std::ceil(needB / 60.9) ? 59 : 61;
  double haveB = 0;
  std::vector<u64> taken = c->Q;
  while (haveB < needB) {
    if ((int)c->B.size() >= PEPSI_MAXB) {
      delete c;
      return PEPSI_E_PARAM;
    }
    u64 p = hostmath::find_prime(bbits, c->N, taken);
    taken.push_back(p);
    c->B.push_back(p);
    haveB += std::log2((double)p);
  }
  c->kb = (int)c->B.size();
  // MAC partial sums (Karatsuba form, S0 = sum cl xl, S2 = sum ch xh and
  // the middle term S1 = sum cl xh + ch xl recovered from SM mod 2^64, so SM
  // itself may wrap): a term of S0, S1 or S2 is below 2^max(bits+1, 2s), and
  // 2^(63 - that) terms plus the residue a fold leaves fit in 64 bits
  {
    int worst = 0;
    for (u64 q : c->Q) {
      const int bits = 64 - __builtin_clzll(q), sp = (bits + 1) / 2;
      worst = std::max(worst, std::max(bits + 1, 2 * sp));
    }
    c->mac_fold = 1 << std::min(20, 63 - worst);
  }
  // roots and tables: Q primes, B primes, then t
  std::vector<u64> all = c->Q;
  all.insert(all.end(), c->B.begin(), c->B.end());
  all.push_back(c->t);
  const int np = (int)all.size();
  std::vector<DevPrime> pr(np);
  std::vector<u64> tw((size_t)np * c->N), tws(tw.size()), itw(tw.size()), itws(tw.size());
  for (int i = 0; i < np; ++i) {
    u64 root = hostmath::min_root(all[i], c->N);
    if (i < c->k) c->psi.push_back(root);
    if (i == np - 1) c->psi_t = root;
    pr[i] = hostmath::make_prime(all[i], c->N);
    hostmath::twiddles(all[i], root, c->N, &tw[(size_t)i * c->N], &tws[(size_t)i * c->N], &itw[(size_t)i * c->N],
                       &itws[(size_t)i * c->N]);
  }
  RnsConst rcst;
  hostmath::rns_constants(c->Q, c->B, c->t, &rcst);
  // binomial table for CW unranking: C(n, r), n <= ell, r <= h
  std::vector<u64> binom((size_t)(c->ell + 1) * (c->h + 1));
  for (int n = 0; n <= c->ell; ++n)
    for (int r = 0; r <= c->h; ++r) binom[(size_t)n * (c->h + 1) + r] = hostmath::binom_sat(n, r);
  // circuit constants: scalars -3, -7, 12, 16, (h!)^-1 (centred) and
  // round(Q [v]_t / t) for v = t-1, 2, 60
  std::vector<u64> consts((size_t)CS_COUNT * c->k);
  auto scalar = [&](int slot, i64 z) {
    for (int i = 0; i < c->k; ++i) {
      u64 q = c->Q[i];
      consts[(size_t)slot * c->k + i] = z >= 0 ? (u64)z % q : (q - ((u64)(-z) % q)) % q;
    }
  };
  scalar(CS_M3, -3);
  scalar(CS_M7, -7);
  scalar(CS_P12, 12);
  scalar(CS_P16, 16);
  {
    u64 f = 1;
    for (int i = 2; i <= c->h; ++i) f = hostmath::mulmod(f, i, c->t);
    u64 z = hostmath::invmod(f, c->t);
    scalar(CS_ZINV, z > c->t / 2 ? (i64)z - (i64)c->t : (i64)z);
  }
  hostmath::delta(c->Q, c->t, c->t - 1, &consts[(size_t)CS_D_TM1 * c->k]);
  hostmath::delta(c->Q, c->t, 2, &consts[(size_t)CS_D_2 * c->k]);
  hostmath::delta(c->Q, c->t, 60, &consts[(size_t)CS_D_60 * c->k]);

  // a blocking stream: ordered with the legacy default stream that most callers use
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaStreamCreate(&c->stream);
  if (e == cudaSuccess) e = kernels_init(c->N);
  if (e == cudaSuccess) e = upload((void**)&c->d_pr, pr.data(), pr.size() * sizeof(DevPrime));
  {  // (twiddle, Shoup companion) pairs: one 16-byte load per butterfly group
    std::vector<ulonglong2> twp(tw.size()), itwp(tw.size());
    for (size_t i = 0; i < tw.size(); ++i) {
      twp[i] = make_ulonglong2(tw[i], tws[i]);
      itwp[i] = make_ulonglong2(itw[i], itws[i]);
    }
    if (e == cudaSuccess) e = upload((void**)&c->d_twp, twp.data(), twp.size() * sizeof(ulonglong2));
    if (e == cudaSuccess) e = upload((void**)&c->d_itwp, itwp.data(), itwp.size() * sizeof(ulonglong2));
  }
  if (e == cudaSuccess) e = upload((void**)&c->d_rc, &rcst, sizeof(rcst));
  if (e == cudaSuccess) e = upload((void**)&c->d_binom, binom.data(), binom.size() * 8);
  if (e == cudaSuccess) e = upload((void**)&c->d_consts, consts.data(), consts.size() * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_s, c->N);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_s_ntt, (size_t)c->k * c->N * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_rlk, (size_t)c->k * 2 * c->k * c->N * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pepsi_destroy(c);
    return cuda_status(e);
  }
  c->V.N = c->N;
  c->V.logN = c->logN;
  c->V.k = c->k;
  c->V.kb = c->kb;
  c->V.tidx = c->k + c->kb;
  c->V.pr = c->d_pr;
  c->V.twp = c->d_twp;
  c->V.itwp = c->d_itwp;
  c->V.rc = c->d_rc;
  for (int i = 0; i < c->k + c->kb; ++i) c->rargs.pr[i] = pr[i];
  c->rargs.rc = rcst;
  c->rargs.N = c->N;
  c->rargs.k = c->k;
  c->rargs.kb = c->kb;
  c->V.host_args = &c->rargs;
  {
    Prof p(c, PC_CLIENT, c->stream, 3);
    launch_keygen(c->V, key_seed, c->d_s, c->d_s_ntt, c->d_rlk, c->stream);
  }
  e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    pepsi_destroy(c);
    return cuda_status(e);
  }
  *out = c;
  return PEPSI_OK;
}

int pepsi_get_info(const pepsi_ctx* c, pepsi_info* info) {
  if (!c || !info) return PEPSI_E_PARAM;
  memset(info, 0, sizeof(*info));
  info->N = c->N;
  info->k = c->k;
  info->kb = c->kb;
  info->ell = c->ell;
  info->h = c->h;
  info->mu = c->prm.mu;
  info->lambda_bar = c->prm.lambda_bar;
  info->logb = c->logN;
  info->t = c->t;
  for (int i = 0; i < c->k; ++i) {
    info->q[i] = c->Q[i];
    info->psi[i] = c->psi[i];
  }
  for (int j = 0; j < c->kb && j < 12; ++j) info->b_primes[j] = c->B[j];
  info->psi_t = c->psi_t;
  info->log2_q = c->log2q;
  info->rescale_group = c->prm.rescale_group;
  info->rescale_cap = c->rescale_cap;
  info->response_primes = (uint32_t)c->resp;
  info->bins = c->blocks * (uint32_t)c->N;
  info->blocks = c->blocks;
  info->plaintext_bytes = c->p7 ? 7 : 8;
  info->gamma = c->gamma;
  return PEPSI_OK;
}

int pepsi_request_bits(uint32_t lambda_bar, uint32_t h, uint64_t bins, double* bits, uint64_t* ell,
                       uint32_t* log2_n, uint32_t* log2_q) {
  u32 ln = 0, lq = 0;
  if (!bits || bins == 0 || lambda_bar == 0 || lambda_bar > 62 || !hostmath::table3(h, &ln, &lq))
    return PEPSI_E_PARAM;
  const u64 l = hostmath::code_length_any(lambda_bar, h);
  if (!l) return PEPSI_E_PARAM;
  const u64 N = 1ull << ln;
  const u64 blocks = (bins + N - 1) / N;
  *bits = (double)blocks * (double)l * (double)N * (double)lq;
  if (ell) *ell = l;
  if (log2_n) *log2_n = ln;
  if (log2_q) *log2_q = lq;
  return PEPSI_OK;
}

int pepsi_comm_optimal_h(uint32_t lambda_bar, uint64_t bins, uint32_t h_max, uint32_t* h) {
  if (!h || h_max == 0 || h_max > 64) return PEPSI_E_PARAM;
  double best = 0;
  u32 arg = 0;
  for (u32 w = 1; w <= h_max; ++w) {
    double b = 0;
    const int rc = pepsi_request_bits(lambda_bar, w, bins, &b, nullptr, nullptr, nullptr);
    if (rc) return rc;
    if (!arg || b < best) {  // strict: a tie keeps the smaller weight
      best = b;
      arg = w;
    }
  }
  *h = arg;
  return PEPSI_OK;
}

int pepsi_set_rescale_group(pepsi_ctx* c, uint32_t rescale_group) {
  if (!c) return PEPSI_E_PARAM;
  c->prm.rescale_group = rescale_group;
  return PEPSI_OK;
}

int pepsi_get_schedule(const pepsi_ctx* c, pepsi_schedule* out) {
  if (!c || !out) return PEPSI_E_PARAM;
  out->chunk = (uint32_t)c->chunk;
  out->ntt_threads = (uint32_t)c->V.nt;
  out->relin_fused = c->relin_fused ? 1u : 0u;
  out->batch_points = (uint32_t)c->batch_points;
  out->batch_groups = (uint32_t)c->batch_groups;
  out->batch_requests = (uint32_t)c->batch_requests;
  return PEPSI_OK;
}

int pepsi_set_schedule(pepsi_ctx* c, const pepsi_schedule* s) {
  if (!c || !s || s->chunk < 1 || s->chunk > 4096 || s->relin_fused > 1) return PEPSI_E_PARAM;
  const u32 nt = s->ntt_threads;
  if (nt && (nt < 64 || nt > 1024 || (nt & (nt - 1)))) return PEPSI_E_PARAM;
  if (s->batch_points != 0 && s->batch_points != 32 && s->batch_points != 64) return PEPSI_E_PARAM;
  if (s->batch_groups > 2 || s->batch_requests > (uint32_t)PEPSI_MAC_MAX_REQUESTS) return PEPSI_E_PARAM;
  c->chunk = (int)s->chunk;
  c->batch_points = s->batch_points ? (int)s->batch_points : 32;
  c->batch_groups = s->batch_groups ? (int)s->batch_groups : 2;
  c->batch_requests = s->batch_requests ? (int)s->batch_requests : 2;
  c->V.nt = (int)nt;
  c->relin_fused = s->relin_fused != 0;
  return PEPSI_OK;
}

namespace {
// Device side of one block: its table [mu][N] (and values) to codeword
// positions, value plaintexts, and the resident prefix of mu_res layers of
// NTT-form plaintexts.
int load_block(pepsi_ctx* c, std::vector<u64>&& hT, std::vector<uint32_t>* hV, u32 mu, u32 mu_res, int* internal) {
  ServerSet S;
  S.mu = mu;
  S.hT = std::move(hT);
  const size_t N = c->N, k = c->k;
  cudaError_t e = upload((void**)&S.dT, S.hT.data(), (size_t)mu * N * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&S.dpos, (size_t)mu * N * c->h * sizeof(uint16_t));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_set(S);
    return cuda_status(e);
  }
  {
    Prof p(c, PC_PTGEN, c->stream);
    launch_cw_unrank(S.dT, (size_t)mu * N, c->d_binom, c->ell, c->h, S.dpos, c->stream);
  }
  if (hV) {  // value plaintexts val_s[layer] (Algorithms 4-5), NTT form over Q u B
    S.has_values = true;
    S.hV = std::move(*hV);
    u32* dv = nullptr;
    e = upload((void**)&dv, S.hV.data(), (size_t)mu * N * sizeof(u32));
    if (e == cudaSuccess) e = cudaMalloc((void**)&S.dVP, (size_t)mu * (c->k + c->kb) * N * 8);
    if (e == cudaSuccess) {
      Prof p(c, PC_PTGEN, c->stream);
      launch_valgen(c->V, dv, (int)mu, S.dVP, c->stream);
      e = cudaStreamSynchronize(c->stream);
    }
    cudaFree(dv);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_set(S);
      return cuda_status(e);
    }
  }
  const size_t per_layer = (size_t)c->ell * k * N;  // plaintext words of a layer
  S.mu_res = mu_res;
  if (S.mu_res) {
    u64* tmp = nullptr;  // split-format words of a few layers, before packing
    int G = 64;          // layers per generation launch
    e = cudaMalloc(&S.dP, (size_t)S.mu_res * per_layer * (c->p7 ? 7 : 8));
    if (e == cudaSuccess && c->p7) {
      G = (int)std::max<size_t>(1, std::min<size_t>(64, ((size_t)1 << 30) / (per_layer * 8)));
      e = cudaMalloc((void**)&tmp, (size_t)G * per_layer * 8);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(S.dP);
      S.dP = nullptr;
      S.mu_res = 0;
    } else {
      S.p7 = c->p7;
      const PlainTab T = S.plain(k * N, c->ell);
      for (u32 l0 = 0; l0 < S.mu_res; l0 += G) {
        const int L = (int)std::min<u32>(G, S.mu_res - l0);
        const size_t off = (size_t)l0 * per_layer;
        Prof p(c, PC_PTGEN, c->stream);
        if (!S.p7) {
          launch_ptgen(c->V, S.dpos + (size_t)l0 * N * c->h, L, c->ell, c->h, static_cast<u64*>(S.dP) + off,
                       c->stream);
        } else {
          launch_ptgen(c->V, S.dpos + (size_t)l0 * N * c->h, L, c->ell, c->h, tmp, c->stream);
          launch_pack7(c->V, tmp, (size_t)L * per_layer, const_cast<u32*>(T.a) + off,
                       const_cast<uint16_t*>(T.b) + off, const_cast<uint8_t*>(T.c) + off, c->stream);
        }
      }
    }
    if (tmp) {
      const cudaError_t e2 = cudaStreamSynchronize(c->stream);
      cudaFree(tmp);
      if (e2 != cudaSuccess) e = e2;
    }
  }
  e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    free_set(S);
    return cuda_status(e);
  }
  S.live = true;
  c->sets.push_back(std::move(S));
  *internal = (int)c->sets.size() - 1;
  return PEPSI_OK;
}

// with_values: the set carries values[n] (labelled PSI / PSI-Sum)
int server_load_impl(pepsi_ctx* c, const uint64_t* items, bool with_values, const uint32_t* values, size_t n,
                     int* set_id) {
  if (!c || (!items && n) || !set_id || (with_values && !values && n)) return PEPSI_E_PARAM;
  if (with_values)
    for (size_t i = 0; i < n; ++i)
      if (values[i] >= c->t) return PEPSI_E_PARAM;
  const size_t N = c->N, bins = (size_t)c->blocks * N;
  hostmath::Hasher H(c->prm.hash_key, c->prm.lambda_bar, c->logb);
  const u32 mu = c->prm.mu ? c->prm.mu : hostmath::mu_rule(n, (u32)bins);
  SetGroup G;
  G.mu = mu;
  G.has_values = with_values;
  u32 maxload = 0;
  int rc = hostmath::simple_hash(H, items, n, mu, G.hT, &maxload, values, with_values ? &G.hV : nullptr);
  if (rc) return rc;
  // resident NTT-form plaintexts: the longest prefix of layers the budget
  // holds for every block
  const size_t per_layer = (size_t)c->ell * c->k * N * (c->p7 ? 7 : 8) * c->blocks;
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  const u64 cap = c->prm.resident_bytes;
  const size_t budget = cap == 0 ? (size_t)(0.6 * (double)freeb) : (cap == UINT64_MAX ? 0 : (size_t)cap);
  const u32 mu_res = (u32)std::min<size_t>(mu, budget / per_layer);
  for (u32 b = 0; b < c->blocks; ++b) {
    std::vector<u64> T((size_t)mu * N);
    std::vector<uint32_t> V(with_values ? (size_t)mu * N : 0);
    for (u32 l = 0; l < mu; ++l) {
      memcpy(&T[(size_t)l * N], &G.hT[(size_t)l * bins + (size_t)b * N], N * 8);
      if (with_values) memcpy(&V[(size_t)l * N], &G.hV[(size_t)l * bins + (size_t)b * N], N * 4);
    }
    int id = -1;
    rc = load_block(c, std::move(T), with_values ? &V : nullptr, mu, mu_res, &id);
    if (rc) {
      for (int i : G.blk) free_set(c->sets[i]);
      return rc;
    }
    G.blk.push_back(id);
  }
  if (c->prof) prof_collect(c);
  G.live = true;
  c->groups.push_back(std::move(G));
  *set_id = (int)c->groups.size() - 1;
  return PEPSI_OK;
}

// Words per block of a request and of a response.
size_t request_block_words(const pepsi_ctx* c) { return (size_t)c->ell * 2 * c->k * c->N; }
size_t response_block_words(const pepsi_ctx* c) { return (size_t)2 * c->resp * c->N; }

// The caller's set, or null.
SetGroup* group(pepsi_ctx* c, int set_id) {
  if (!c || set_id < 0 || set_id >= (int)c->groups.size() || !c->groups[set_id].live) return nullptr;
  return &c->groups[set_id];
}
}  // namespace

int pepsi_server_load(pepsi_ctx* c, const uint64_t* items, size_t n, int* set_id) {
  return server_load_impl(c, items, false, nullptr, n, set_id);
}

int pepsi_server_load_values(pepsi_ctx* c, const uint64_t* items, const uint32_t* values, size_t n, int* set_id) {
  return server_load_impl(c, items, true, values, n, set_id);
}

int pepsi_server_values(pepsi_ctx* c, int set_id, uint32_t* out) {
  SetGroup* G = group(c, set_id);
  if (!G || !out || !G->has_values) return PEPSI_E_PARAM;
  memcpy(out, G->hV.data(), G->hV.size() * sizeof(uint32_t));
  return PEPSI_OK;
}

int pepsi_server_table(pepsi_ctx* c, int set_id, uint64_t* out) {
  SetGroup* G = group(c, set_id);
  if (!G || !out) return PEPSI_E_PARAM;
  memcpy(out, G->hT.data(), G->hT.size() * 8);
  return PEPSI_OK;
}

int pepsi_server_plaintexts(pepsi_ctx* c, int set_id, uint32_t layer0, uint32_t nl, uint64_t* out, void* stream) {
  SetGroup* G = group(c, set_id);
  if (!G || !out || (u64)layer0 + nl > G->mu) return PEPSI_E_PARAM;
  cudaStream_t st = pick(c, stream);
  const size_t per = (size_t)c->ell * c->k * c->N;
  cudaError_t e = cudaSuccess;
  u64* tmp = (u64*)scratch(c, S_PC, (size_t)nl * per * 8, &e);
  if (!tmp) return cuda_status(e);
  for (size_t b = 0; b < G->blk.size(); ++b) {
    ServerSet& S = c->sets[G->blk[b]];
    if ((u64)layer0 + nl <= S.mu_res && S.p7) {  // the stored planes, put back together
      const PlainTab T = S.plain((size_t)c->k * c->N, c->ell, layer0);
      launch_unpack7(T.a, T.b, T.c, (size_t)nl * per, tmp, st);
    } else {
      if ((u64)layer0 + nl <= S.mu_res) {
        CKS(cudaMemcpyAsync(tmp, static_cast<const u64*>(S.dP) + (size_t)layer0 * per, (size_t)nl * per * 8,
                            cudaMemcpyDeviceToDevice, st));
      } else {
        Prof p(c, PC_PTGEN, st);
        launch_ptgen(c->V, S.dpos + (size_t)layer0 * c->N * c->h, nl, c->ell, c->h, tmp, st);
      }
      launch_split(c->V, tmp, (size_t)nl * c->ell, false, st);  // stored split; returned reduced
    }
    e = copy_any(out + b * nl * per, tmp, (size_t)nl * per * 8, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return PEPSI_OK;
}

namespace {
// scratch id of the device cuckoo placement's state
constexpr int kScratchCuckoo = 51;

// The client's cuckoo placement in parallel rounds on the device (see
// pepsi_params.client_cuckoo): table [bins][gamma] of x_L values (dummies
// PEPSI_DUMMY) and where[u] = bin * gamma + slot, as hostmath::cuckoo.
int device_cuckoo(pepsi_ctx* c, const hostmath::Hasher& H, const u64* items, size_t m, std::vector<u64>& table,
                  std::vector<int32_t>& where, cudaStream_t st) {
  const u32 nbins = 1u << c->logb, g = c->gamma;
  const size_t cells = (size_t)nbins * g;
  if (m > cells || m > 0x7FFFFFFFu) return PEPSI_E_CUCKOO_FAIL;
  std::vector<u64> xl(m);
  std::vector<u32> bins3(3 * m);
  for (size_t u = 0; u < m; ++u) H(items[u], &xl[u], &bins3[3 * u]);
  // one buffer: bins3 | claim | slot_item | load | evictions | unplaced | state | choice
  const size_t o_claim = 3 * m, o_slot = o_claim + nbins, o_load = o_slot + cells, o_ev = o_load + nbins,
               o_cnt = o_ev + nbins, words = o_cnt + 1;
  cudaError_t e = cudaSuccess;
  u32* d = (u32*)scratch(c, kScratchCuckoo, words * 4 + 2 * m + 16, &e);
  if (!d) return cuda_status(e);
  uint8_t* state = reinterpret_cast<uint8_t*>(d + words);
  uint8_t* choice = state + m;
  CKS(cudaMemcpyAsync(d, bins3.data(), 3 * m * 4, cudaMemcpyHostToDevice, st));
  CKS(cudaMemsetAsync(d + o_claim, 0xFF, (nbins + cells) * 4, st));  // no claims, free slots (-1)
  CKS(cudaMemsetAsync(d + o_load, 0, 2 * (size_t)nbins * 4, st));
  CKS(cudaMemsetAsync(state, 1, m, st));
  CKS(cudaMemsetAsync(choice, 0, m, st));
  u32 left = (u32)m;
  // rounds in groups of four between reads of the count (a round with
  // nothing unplaced changes nothing), at most 1000
  for (int r = 0; r < 1000 && left; r += 4) {
    for (int i = 0; i < 4; ++i) {
      CKS(cudaMemsetAsync(d + o_cnt, 0, 4, st));
      launch_cuckoo_round(d, (u32)m, nbins, g, d + o_claim, reinterpret_cast<int32_t*>(d + o_slot), d + o_load,
                          d + o_ev, state, choice, d + o_cnt, st);
    }
    CKS(cudaMemcpyAsync(&left, d + o_cnt, 4, cudaMemcpyDeviceToHost, st));
    CKS(cudaStreamSynchronize(st));
  }
  if (left) return PEPSI_E_CUCKOO_FAIL;
  std::vector<int32_t> slot(cells);
  CKS(cudaMemcpyAsync(slot.data(), d + o_slot, cells * 4, cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  table.assign(cells, PEPSI_DUMMY);
  where.assign(m, -1);
  for (size_t i = 0; i < cells; ++i)
    if (slot[i] >= 0) {
      table[i] = xl[slot[i]];
      where[slot[i]] = (int32_t)i;
    }
  return PEPSI_OK;
}
}  // namespace

int pepsi_query(pepsi_ctx* c, const uint64_t* items, size_t m, uint64_t enc_seed, uint64_t* cts,
                int32_t* bin_of_item, void* stream) {
  if (!c || (!items && m) || !cts) return PEPSI_E_PARAM;
  cudaStream_t st = pick(c, stream);
  hostmath::Hasher H(c->prm.hash_key, c->prm.lambda_bar, c->logb);
  std::vector<u64> table;  // [bins][gamma]
  std::vector<int32_t> where;
  int rc = c->prm.client_cuckoo ? device_cuckoo(c, H, items, m, table, where, st)
                                 : hostmath::cuckoo(H, items, m, c->gamma, table, where);
  if (rc) return rc;
  if (bin_of_item) memcpy(bin_of_item, where.data(), m * sizeof(int32_t));
  cudaError_t e = cudaSuccess;
  const size_t N = c->N, bins = (size_t)c->blocks * N, g = c->gamma;
  // batch i of the client table: slot i of every bin, laid out [gamma][bins]
  std::vector<u64> batches(bins * g);
  for (size_t bin = 0; bin < bins; ++bin)
    for (size_t i = 0; i < g; ++i) batches[i * bins + bin] = table[bin * g + i];
  u64* dTc = (u64*)scratch(c, S_TC, bins * g * 8, &e);
  uint16_t* dpos = (uint16_t*)scratch(c, S_POS, bins * g * c->h * sizeof(uint16_t), &e);
  const size_t words = request_block_words(c) * c->blocks * g;
  const bool dev_out = is_device_ptr(cts);
  u64* dct = dev_out ? cts : (u64*)scratch(c, S_CT, words * 8, &e);
  if (!dTc || !dpos || !dct) return cuda_status(e);
  CKS(copy_any(dTc, batches.data(), bins * g * 8, st));
  {
    Prof p(c, PC_CLIENT, st);
    launch_cw_unrank(dTc, bins * g, c->d_binom, c->ell, c->h, dpos, st);
  }
  for (u32 b = 0; b < c->blocks; ++b)  // ciphertexts of (block b, batch i): (b * gamma + i) * ell ...
    for (size_t i = 0; i < g; ++i) {
      const size_t r = (size_t)b * g + i;
      Prof p(c, PC_CLIENT, st);
      launch_encrypt(c->V, dpos + (i * bins + (size_t)b * N) * c->h, c->ell, c->h, c->d_s_ntt, enc_seed,
                     (u64)r * c->ell, dct + r * request_block_words(c), st);
    }
  if (!dev_out) CKS(copy_any(cts, dct, words * 8, st));
  e = cudaStreamSynchronize(st);  // the host tables must outlive the copies
  if (e == cudaSuccess) e = cudaGetLastError();
  if (c->prof) prof_collect(c);
  return cuda_status(e);
}

int pepsi_eval(pepsi_ctx* c, int set_id, const uint64_t* cts, int mode, uint64_t mask_seed, uint64_t* out_ct,
               void* stream) {
  SetGroup* G = group(c, set_id);
  if (!G || !out_ct || !cts) return PEPSI_E_PARAM;
  cudaStream_t st = pick(c, stream);
  if (c->gamma == 1) {
    for (size_t b = 0; b < G->blk.size(); ++b) {  // block b: its request block, mask seed + b
      const int rc = eval_core(c, G->blk[b], cts + b * request_block_words(c), 0, G->mu, mode, mask_seed + b,
                               out_ct + b * response_block_words(c), nullptr, nullptr, st);
      if (rc) return rc;
    }
    return PEPSI_OK;
  }
  // gamma client batches per block (Algorithm 2's outer loop): the batches of a
  // block are requests on the same internal set, evaluated together
  std::vector<int> ids, md;
  std::vector<const u64*> in;
  std::vector<u64*> out;
  std::vector<u64> seeds;
  for (size_t b = 0; b < G->blk.size(); ++b)
    for (size_t i = 0; i < c->gamma; ++i) {
      const size_t r = b * c->gamma + i;
      ids.push_back(G->blk[b]);
      in.push_back(cts + r * request_block_words(c));
      out.push_back(out_ct + r * response_block_words(c));
      md.push_back(mode);
      seeds.push_back(mask_seed + r);
    }
  return eval_batch_core(c, (int)ids.size(), ids.data(), in.data(), md.data(), seeds.data(), out.data(), st);
}

int pepsi_autotune(pepsi_ctx* c, int set_id, const uint64_t* cts, void* stream, uint32_t* chosen) {
  SetGroup* G = group(c, set_id);
  if (!G || !cts) return PEPSI_E_PARAM;
  cudaStream_t st = pick(c, stream);
  cudaError_t e = cudaSuccess;
  u64* out = (u64*)scratch(c, kScratchTune, response_block_words(c) * c->blocks * c->gamma * 8, &e);
  if (!out) return cuda_status(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CKS(cudaEventCreate(&e0));
  CKS(cudaEventCreate(&e1));
  const pepsi_schedule saved{(uint32_t)c->chunk, (uint32_t)c->V.nt, c->relin_fused ? 1u : 0u,
                             (uint32_t)c->batch_points, (uint32_t)c->batch_groups, (uint32_t)c->batch_requests};
  // ms of two evaluations after a warm-up under the current schedule (< 0: error code)
  auto time_it = [&](float* ms) -> int {
    int rc = PEPSI_OK;
    for (int rep = 0; rep < 3 && !rc; ++rep) {
      if (rep == 1) cudaEventRecord(e0, st);
      rc = pepsi_eval(c, set_id, cts, PEPSI_MODE_INDICATOR, 0, out, st);
    }
    if (rc) return rc;
    cudaEventRecord(e1, st);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(ms, e0, e1);
    return ce == cudaSuccess ? PEPSI_OK : cuda_status(ce);
  };
  // circuit scratch per layer of a chunk: the pipeline's buffers (eval_bufs)
  const size_t kN = (size_t)c->k * c->N, kbN = (size_t)c->kb * c->N;
  const size_t per_layer = (24 * kN + 7 * kbN) * 8;
  const size_t scratch_cap = (size_t)4 << 30;
  int rc = PEPSI_OK;
  float best_ms = 0;
  // 1: the layer chunk (larger chunks fill the GPU with more blocks per
  // launch), as the balanced size an evaluation of the set's mu layers uses
  int best_chunk = c->chunk, last = 0;
  for (int want : {32, 64, 128, 256, 512, 1024, 2048, 4096}) {
    const int chunk = balanced_chunk(want, G->mu);
    if (chunk == last) continue;
    last = chunk;
    if (want > 32 && (size_t)chunk * per_layer > scratch_cap) break;
    c->chunk = chunk;
    float ms = 0;
    rc = time_it(&ms);
    if (rc == PEPSI_E_NOMEM && best_ms > 0) {  // this chunk's scratch does not fit: keep the best so far
      cudaGetLastError();
      rc = PEPSI_OK;
      break;
    }
    if (rc) break;
    if (best_ms == 0 || ms < best_ms) {
      best_ms = ms;
      best_chunk = chunk;
    }
    if ((u32)chunk >= G->mu) break;  // one chunk holds every layer
  }
  c->chunk = best_chunk;
  // 2: threads per transform block (the default, half and twice it)
  if (!rc) {
    const int def = c->N >= 16384 ? 1024 : std::max(32, std::min(512, c->N / 8));
    int best_nt = 0;
    for (int nt : {def / 2, def * 2}) {
      if (nt < 64 || nt > 1024) continue;
      c->V.nt = nt;
      float ms = 0;
      rc = time_it(&ms);
      if (rc) break;
      if (ms < best_ms) {
        best_ms = ms;
        best_nt = nt;
      }
    }
    c->V.nt = best_nt;
  }
  // 3: the relinearisation feeding the affine step: fused with its transform, or stored
  if (!rc && (c->h == 4 || c->h == 8)) {
    c->relin_fused = false;
    float ms = 0;
    rc = time_it(&ms);
    if (!rc && ms < best_ms) best_ms = ms;
    else c->relin_fused = true;
  }
  // 4: requests per shared multiply-accumulate, on a batch of four copies of the request
  if (!rc && G->blk.size() == 1 && c->gamma == 1) {
    std::vector<u64*> outs(4, nullptr);
    u64* ob = (u64*)scratch(c, kScratchTuneBatch, 4 * response_block_words(c) * 8, &e);
    if (!ob) rc = cuda_status(e);
    for (int i = 0; i < 4 && !rc; ++i) outs[i] = ob + (size_t)i * response_block_words(c);
    const int ids[4] = {set_id, set_id, set_id, set_id};
    const u64* in[4] = {cts, cts, cts, cts};
    float best_b = 0;
    int best_r = c->batch_requests, best_g = c->batch_groups;
    const int cand[5][2] = {{1, 2}, {2, 2}, {2, 1}, {4, 2}, {4, 1}};  // (requests, warp groups)
    for (const auto& rg : cand) {
      if (rc) break;
      const int br = rg[0];
      c->batch_requests = br;
      c->batch_groups = rg[1];
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        rc = pepsi_eval_batch(c, 4, ids, in, nullptr, nullptr, outs.data(), st);
      }
      if (rc) break;
      cudaEventRecord(e1, st);
      float ms = 0;
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) {
        rc = cuda_status(ce);
        break;
      }
      if (best_b == 0 || ms < best_b) {
        best_b = ms;
        best_r = br;
        best_g = rg[1];
      }
    }
    c->batch_requests = best_r;
    c->batch_groups = best_g;
    // the batch buffers served only the timing: four requests' prepared
    // words, h' and sums, twice, are not kept for evaluations that may
    // never batch
    for (int id : {(int)S_CB, (int)S_CB2, (int)S_HB, (int)S_HB2, (int)S_ACCB, (int)S_ACCXB, kScratchTuneBatch})
      scratch_release(c, id);
  }
  if (rc) {
    c->chunk = (int)saved.chunk;
    c->V.nt = (int)saved.ntt_threads;
    c->relin_fused = saved.relin_fused != 0;
    c->batch_requests = (int)saved.batch_requests;
    c->batch_groups = (int)saved.batch_groups;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc && chosen) *chosen = (uint32_t)c->chunk;
  return rc;
}

int pepsi_eval_batch(pepsi_ctx* c, int nq, const int* set_ids, const uint64_t* const* cts, const int* modes,
                     const uint64_t* mask_seeds, uint64_t* const* out_cts, void* stream) {
  if (!c || nq < 0 || (nq && (!set_ids || !cts || !out_cts))) return PEPSI_E_PARAM;
  if (!nq) return PEPSI_OK;
  // one internal request per (request, block)
  std::vector<int> ids, md;
  std::vector<const u64*> in;
  std::vector<u64*> out;
  std::vector<u64> seeds;
  for (int i = 0; i < nq; ++i) {
    SetGroup* G = group(c, set_ids[i]);
    if (!G || !cts[i] || !out_cts[i]) return PEPSI_E_PARAM;
    for (size_t b = 0; b < G->blk.size(); ++b)
      for (size_t j = 0; j < c->gamma; ++j) {  // (block b, client batch j)
        const size_t r = b * c->gamma + j;
        ids.push_back(G->blk[b]);
        in.push_back(cts[i] + r * request_block_words(c));
        out.push_back(out_cts[i] + r * response_block_words(c));
        md.push_back(modes ? modes[i] : PEPSI_MODE_INDICATOR);
        seeds.push_back((mask_seeds ? mask_seeds[i] : 0) + r);
      }
  }
  return eval_batch_core(c, (int)ids.size(), ids.data(), in.data(), md.data(), seeds.data(), out.data(),
                         pick(c, stream));
}

int pepsi_eval_layers(pepsi_ctx* c, int set_id, const uint64_t* cts, uint32_t layer0, uint32_t nl, uint64_t* h_out,
                      uint64_t* e_out, void* stream) {
  SetGroup* G = group(c, set_id);
  if (!G || nl == 0 || !cts) return PEPSI_E_PARAM;
  const size_t kN = (size_t)c->k * c->N;
  cudaStream_t st = pick(c, stream);
  for (size_t b = 0; b < G->blk.size(); ++b)
    for (size_t i = 0; i < c->gamma; ++i) {  // (block b, client batch i)
      const size_t r = b * c->gamma + i;
      const int rc = eval_core(c, G->blk[b], cts + r * request_block_words(c), layer0, nl, PEPSI_MODE_INDICATOR,
                               0, nullptr, h_out ? h_out + r * nl * 2 * kN : nullptr,
                               e_out ? e_out + r * nl * 3 * kN : nullptr, st);
      if (rc) return rc;
    }
  return PEPSI_OK;
}

int pepsi_decrypt_primes(pepsi_ctx* c, const uint64_t* ct, uint32_t nprimes, uint32_t* slots,
                         double* noise_budget_bits) {
  if (!c || !ct || !slots || nprimes == 0 || nprimes > (uint32_t)c->k) return PEPSI_E_PARAM;
  const int r = (int)nprimes;
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  const size_t N = c->N, ct2 = 2 * (size_t)r * N;
  u64* din = (u64*)scratch(c, S_IN, ct2 * 8, &e);
  u64* z = (u64*)scratch(c, S_DEC_Z, (size_t)r * N * 8, &e);
  u32* m = (u32*)scratch(c, S_DEC_M, N * 4, &e);
  u32* sl = (u32*)scratch(c, S_DEC_SLOTS, N * 4, &e);
  unsigned long long* mx = (unsigned long long*)scratch(c, S_DEC_MAX, 8, &e);
  if (!din || !z || !m || !sl || !mx) return cuda_status(e);
  CKS(copy_any(din, ct, ct2 * 8, st));
  // the same tables, viewed as the first r primes, with the constants of Q_r
  const RnsArgs& A = sub_args(c, r);
  DevView Vr = c->V;
  Vr.k = r;
  Vr.host_args = &A;
  {
    Prof p(c, PC_CLIENT, st, 3);
    launch_decrypt(Vr, din, c->d_s_ntt, z, m, sl, mx, st);
  }
  unsigned long long bits = 0;
  CKS(cudaMemcpyAsync(slots, sl, N * 4, cudaMemcpyDeviceToHost, st));
  CKS(cudaMemcpyAsync(&bits, mx, 8, cudaMemcpyDeviceToHost, st));
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  if (c->prof) prof_collect(c);
  double maxr, log2qr = 0;
  memcpy(&maxr, &bits, 8);
  for (int i = 0; i < r; ++i) log2qr += std::log2((double)c->Q[i]);
  const double budget = maxr > 0 ? log2qr - 1.0 - std::log2(maxr) : INFINITY;
  if (noise_budget_bits) *noise_budget_bits = budget;
  return budget > 0 ? PEPSI_OK : PEPSI_E_NOISE;
}

int pepsi_decrypt(pepsi_ctx* c, const uint64_t* ct, uint32_t* slots, double* noise_budget_bits) {
  if (!c) return PEPSI_E_PARAM;
  return pepsi_decrypt_primes(c, ct, (uint32_t)c->k, slots, noise_budget_bits);
}

int pepsi_mod_switch(pepsi_ctx* c, const uint64_t* ct, size_t n, uint32_t nprimes, uint64_t* out, void* stream) {
  if (!c || !ct || !out || nprimes == 0 || nprimes > (uint32_t)c->k) return PEPSI_E_PARAM;
  if (!n) return PEPSI_OK;
  cudaStream_t st = pick(c, stream);
  const size_t N = c->N, r = nprimes;
  const size_t in_w = n * 2 * c->k * N, out_w = n * 2 * r * N;
  if ((int)r == c->k) {
    CKS(copy_any(out, ct, in_w * 8, st));
  } else {
    cudaError_t e = cudaSuccess;
    const bool din = is_device_ptr(ct), dout = is_device_ptr(out);
    const u64* src = ct;
    u64* dst = out;
    if (!din) {
      u64* b = (u64*)scratch(c, S_CT, in_w * 8, &e);
      if (!b) return cuda_status(e);
      CKS(copy_any(b, ct, in_w * 8, st));
      src = b;
    }
    if (!dout) {
      dst = (u64*)scratch(c, S_TC, out_w * 8, &e);
      if (!dst) return cuda_status(e);
    }
    {
      Prof p(c, PC_CLIENT, st);
      launch_modswitch(c->V, ms_args(c, (int)r), src, dst, n, st);
    }
    if (!dout) CKS(copy_any(out, dst, out_w * 8, st));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  if (!is_device_ptr(out)) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return PEPSI_OK;
}

int pepsi_ntt(pepsi_ctx* c, uint64_t* polys, size_t count, int inverse, void* stream) {
  if (!c || !polys) return PEPSI_E_PARAM;
  if (!count) return PEPSI_OK;
  if (!is_device_ptr(polys)) return PEPSI_E_PARAM;
  cudaStream_t st = pick(c, stream);
  const size_t kN = (size_t)c->k * c->N;
  ntt(c, !inverse, polys, polys, count, c->k, 0, kN, kN, st);
  return cuda_status(cudaGetLastError());
}

int pepsi_ct_mult(pepsi_ctx* c, const uint64_t* a, const uint64_t* b, size_t n, int relin_flag, uint64_t* out,
                  void* stream) {
  if (!c || !a || !b || !out) return PEPSI_E_PARAM;
  if (!n) return PEPSI_OK;
  if (!is_device_ptr(a) || !is_device_ptr(b) || !is_device_ptr(out)) return PEPSI_E_PARAM;
  cudaStream_t st = pick(c, stream);
  const size_t k = c->k, kb = c->kb, N = c->N, np = k + kb;
  const size_t kN = k * N, kbN = kb * N;
  cudaError_t e = cudaSuccess;
  u64* AQ = (u64*)scratch(c, S_U, n * 2 * kN * 8, &e);
  u64* BQ = (u64*)scratch(c, S_W, n * 2 * kN * 8, &e);
  u64* AB = (u64*)scratch(c, S_XB, n * 2 * kbN * 8, &e);
  u64* BB = (u64*)scratch(c, S_YB, n * 2 * kbN * 8, &e);
  u64* T3 = (u64*)scratch(c, S_T3, n * 3 * np * N * 8, &e);
  u64* D = (u64*)scratch(c, S_D, n * 3 * kN * 8, &e);
  u64* R = (u64*)scratch(c, S_R, n * 2 * kN * 8, &e);
  if (!AQ || !BQ || !AB || !BB || !T3 || !D || !R) return cuda_status(e);
  const int L = (int)n;
  {
    Prof p(c, PC_LIFT, st);
    launch_lift(c->V, a, AB, L, nullptr, nullptr, st);
  }
  {
    Prof p(c, PC_LIFT, st);
    launch_lift(c->V, b, BB, L, nullptr, nullptr, st);
  }
  ntt(c, true, a, AQ, n * 2, c->k, 0, kN, kN, st);
  ntt(c, true, b, BQ, n * 2, c->k, 0, kN, kN, st);
  ntt(c, true, AB, AB, n * 2, c->kb, c->k, kbN, kbN, st);
  ntt(c, true, BB, BB, n * 2, c->kb, c->k, kbN, kbN, st);
  mult_tail(c, AQ, AB, BQ, BB, nullptr, nullptr, false, T3, D, L, st);
  if (relin_flag && c->relin_fused) {
    // the key-switching sum on the load of the inverse NTT (plus 0 * D, the
    // affine step of the circuit with a zero scalar): the same words
    u64* DG = (u64*)scratch(c, kScratchDG, (size_t)L * (k + 2) * kN * 8, &e);
    u64* zero = (u64*)scratch(c, kScratchZeroK, k * 8, &e);
    if (!DG || !zero) return cuda_status(e);
    CKS(cudaMemsetAsync(zero, 0, k * 8, st));
    Prof p(c, PC_RELIN, st, 2);
    launch_relin_digits(c->V, D, DG, L, st);
    launch_relin_axpy_intt(c->V, DG, c->d_rlk, zero, D, R, out, L, st);
  } else if (relin_flag) {
    relin(c, D, R, L, st);
    ntt(c, false, R, out, n * 2, c->k, 0, kN, kN, st);
  } else {
    CKS(cudaMemcpyAsync(out, D, n * 3 * kN * 8, cudaMemcpyDeviceToDevice, st));
  }
  return cuda_status(cudaGetLastError());
}

int pepsi_relin(pepsi_ctx* c, const uint64_t* in, size_t n, uint64_t* out, void* stream) {
  if (!c || !in || !out) return PEPSI_E_PARAM;
  if (!n) return PEPSI_OK;
  if (!is_device_ptr(in) || !is_device_ptr(out)) return PEPSI_E_PARAM;
  cudaStream_t st = pick(c, stream);
  const size_t kN = (size_t)c->k * c->N;
  cudaError_t e = cudaSuccess;
  u64* R = (u64*)scratch(c, S_R, n * 2 * kN * 8, &e);
  if (!R) return cuda_status(e);
  relin(c, in, R, (int)n, st);
  ntt(c, false, R, out, n * 2, c->k, 0, kN, kN, st);
  return cuda_status(cudaGetLastError());
}

int pepsi_relin_noalloc(pepsi_ctx* c, const uint64_t* in, size_t n, uint64_t* out, void* stream) {
  if (!c || !in || !out) return PEPSI_E_PARAM;
  if (!n) return PEPSI_OK;
  const size_t kN = (size_t)c->k * c->N;
  // bytes per ciphertext: (k+2) digit rows and 2 result rows of k*N words;
  // n is checked against the array before any product that could wrap
  const size_t per_ct = (size_t)(c->k + 2 + 2) * kN * sizeof(u64);
  const size_t max_n = (size_t)PEPSI_NOALLOC_SCRATCH_BYTES / per_ct;
  if (n > max_n) {
    g_last_error = "pepsi_relin_noalloc: " + std::to_string(n) + " ciphertexts need " + std::to_string(per_ct) +
                   " bytes of scratch each, the fixed array holds " +
                   std::to_string((size_t)PEPSI_NOALLOC_SCRATCH_BYTES) + " bytes (at most " + std::to_string(max_n) +
                   " ciphertexts)";
    return PEPSI_E_PARAM;
  }
  if (!is_device_ptr(in) || !is_device_ptr(out)) return PEPSI_E_PARAM;
  u64* base = nullptr;
  int rc = noalloc_scratch(c, &base);
  if (rc) return rc;
  const size_t dg_words = n * (size_t)(c->k + 2) * kN;
  u64* DG = base;
  u64* R = base + dg_words;
  cudaStream_t st = pick(c, stream);
  // every word of DG and R is written before it is read: nothing to clear
  launch_relin(c->V, in, c->d_rlk, DG, R, (int)n, st);
  launch_ntt(c->V, false, R, out, n * 2, c->k, 0, kN, kN, st);
  return cuda_status(cudaGetLastError());
}

int pepsi_export_keys(pepsi_ctx* c, int8_t* s, uint64_t* rlk) {
  if (!c) return PEPSI_E_PARAM;
  cudaStream_t st = c->stream;
  const size_t kN = (size_t)c->k * c->N, words = (size_t)c->k * 2 * kN;
  if (s) CKS(cudaMemcpyAsync(s, c->d_s, c->N, cudaMemcpyDeviceToHost, st));
  if (rlk) {
    cudaError_t e = cudaSuccess;
    u64* tmp = (u64*)scratch(c, S_CT, words * 8, &e);
    if (!tmp) return cuda_status(e);
    ntt(c, false, c->d_rlk, tmp, (size_t)c->k * 2, c->k, 0, kN, kN, st);
    CKS(cudaMemcpyAsync(rlk, tmp, words * 8, cudaMemcpyDeviceToHost, st));
  }
  return cuda_status(cudaStreamSynchronize(st));
}

int pepsi_wait_probe(pepsi_ctx* c, int arrive) {
  if (!c) return PEPSI_E_PARAM;
  launch_wait_probe(arrive, c->d_err, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  return take_error_flag(c) ? PEPSI_E_TIMEOUT : PEPSI_OK;
}

int pepsi_int_peak(int form, double* ops_per_s) {
  if (!ops_per_s || form < 0 || form > 2) return PEPSI_E_PARAM;
  *ops_per_s = measure_int_peak(form);
  if (*ops_per_s > 0) return PEPSI_OK;
  const cudaError_t e = cudaGetLastError();
  return cuda_status(e != cudaSuccess ? e : cudaErrorUnknown);
}

int pepsi_profile_enable(pepsi_ctx* c, int on) {
  if (!c) return PEPSI_E_PARAM;
  cudaStreamSynchronize(c->stream);
  prof_collect(c);
  c->prof = on != 0;
  for (int i = 0; i < PC_COUNT; ++i) {
    c->prof_launch[i] = 0;
    c->prof_ms[i] = 0;
  }
  c->launches = 0;
  return PEPSI_OK;
}

int pepsi_profile_read(pepsi_ctx* c, const char** names, uint64_t* launches, double* total_ms, int max) {
  if (!c) return PEPSI_E_PARAM;
  cudaDeviceSynchronize();
  prof_collect(c);
  for (int i = 0; i < PC_COUNT && i < max; ++i) {
    if (names) names[i] = kProfNames[i];
    if (launches) launches[i] = c->prof_launch[i];
    if (total_ms) total_ms[i] = c->prof_ms[i];
  }
  return PC_COUNT;
}

}  // extern "C"
