// Internal declarations shared by the translation units of the library:
// the context, the server sets, the scratch layout of the evaluation
// pipeline and the pipeline's steps (pepsi.cu), used by the request engine
// (engine.cu).  Not part of the C ABI.
#pragma once
#include <algorithm>
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "host.h"
#include "kernels.h"
#include "pepsi.h"

namespace pepsi_detail {

enum ProfClass { PC_NTT, PC_PTGEN, PC_MAC, PC_LIFT, PC_TENSOR, PC_SCALE, PC_RELIN, PC_POINTWISE, PC_CLIENT, PC_COUNT };
inline const char* const kProfNames[PC_COUNT] = {"ntt",         "ptgen", "mac",      "lift",  "tensor",
                                                 "scale_round", "relin", "pointwise", "client"};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct ServerSet {
  bool live = false;
  u32 mu = 0;
  std::vector<u64> hT;          // [mu][N] host copy of T_s
  u64* dT = nullptr;            // [mu][N]
  uint16_t* dpos = nullptr;     // [mu][N][h]
  // resident plaintexts of a prefix of the layers, [mu_res][ell][k][N]: one
  // device array holding either 64-bit words in the split operand format, or
  // (p7) the three planes of the 7-byte format one after another
  void* dP = nullptr;
  bool p7 = false;
  u32 mu_res = 0;               // layers [0, mu_res) resident, the rest regenerated per chunk
  bool has_values = false;      // loaded with values (labelled PSI / PSI-Sum)
  std::vector<uint32_t> hV;     // [mu][N] host copy of the value table
  u64* dVP = nullptr;           // [mu][k+kb][N] value plaintexts val_s, NTT form over Q u B
  // the resident plaintexts as a table for the multiply-accumulate, from layer l0
  PlainTab plain(size_t kN, int ell, u32 l0 = 0) const {
    const size_t words = (size_t)mu_res * ell * kN, off = (size_t)l0 * ell * kN;
    if (!p7) return plain_words(static_cast<const u64*>(dP)).at(off);
    PlainTab t;
    t.a = static_cast<const u32*>(dP);
    t.b = reinterpret_cast<const uint16_t*>(t.a + words);
    t.c = reinterpret_cast<const uint8_t*>(t.b + words);
    return t.at(off);
  }
};

// A server set as the caller sees it: its b = B*N bins are B blocks of N
// slots, each an internal ServerSet (its own layers and plaintexts) that
// is evaluated against the request's block of the same index.
struct SetGroup {
  bool live = false;
  u32 mu = 0;
  std::vector<int> blk;       // internal set of each block
  std::vector<u64> hT;        // [mu][bins] the whole table
  std::vector<uint32_t> hV;   // [mu][bins] values, when loaded with values
  bool has_values = false;
};

}  // namespace pepsi_detail

struct pepsi_ctx {
  pepsi_params prm{};
  int device = 0;  // the CUDA device current at setup: every launch of the context goes there
  bool borrowed = false;  // a lane (ctx_fork): keys, tables and sets belong to the parent
  int N = 0, logN = 0, k = 0, kb = 0, ell = 0, h = 0;
  u64 t = 0;
  std::vector<u64> Q, B, psi;
  u64 psi_t = 0;
  double log2q = 0;
  DevView V{};
  RnsArgs rargs{};  // host copy of the by-value RNS kernel parameters
  cudaStream_t stream = nullptr;
  cudaStream_t aux_stream = nullptr;  // overlapped multiply-accumulates of pepsi_eval_batch
  cudaEvent_t aux_ev[4] = {};
  // host requests: copies of the request pieces, overlapped with the
  // multiply-accumulate of the pieces already on the device (two pieces, the
  // first short: each further MAC launch costs its pipeline fill, measured to
  // outweigh the copy it hides)
  static constexpr int kPieces = 2;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ready = nullptr, copy_ev[kPieces] = {};
  // device tables and keys
  DevPrime* d_pr = nullptr;
  ulonglong2 *d_twp = nullptr, *d_itwp = nullptr;  // twiddles interleaved with their Shoup companions
  RnsConst* d_rc = nullptr;
  u64* d_binom = nullptr;
  int8_t* d_s = nullptr;
  u64* d_s_ntt = nullptr;  // [k][N]
  u64* d_rlk = nullptr;    // [k][2][k][N] NTT form
  u64* d_consts = nullptr; // residues of circuit scalars and constants, [slot][k]
  int* d_err = nullptr;     // set by kernels whose bounded wait expired
  int mac_fold = 1;         // terms between folds of the MAC partial sums
  std::vector<pepsi_detail::ServerSet> sets;   // internal: one per block of a loaded set
  std::vector<pepsi_detail::SetGroup> groups;  // the caller's set ids
  u32 logb = 0, blocks = 1;      // bins = blocks * N = 2^logb
  u32 gamma = 1;                 // client maximum bin load: client batches per block
  // scratch, grown on demand
  std::vector<pepsi_detail::DevBuf> scratch;
  int chunk = 64;  // layers per circuit chunk (pepsi_autotune may change it)
  bool relin_fused = true;  // key-switching sum on the load of the affine step's inverse NTT
  int batch_points = 32;    // points per block of the multi-request multiply-accumulate
  int batch_groups = 2;     // warp groups of the multi-request multiply-accumulate
  int batch_requests = 2;   // most requests per shared multiply-accumulate launch
  u32 rescale_cap = 1;      // most layers one rounding of the last products may cover
  bool value_margin = false;  // B also holds the value products under lazy rescaling
  int resp = 0;               // primes of the evaluation's response (k: no switching)
  bool p7 = false;            // resident plaintexts in the 7-byte format
  // per prime count r < k: modulus-switching constants and the RNS
  // constants of Q_r for decryption, built on first use
  std::unique_ptr<ModSwitchArgs> ms_args[PEPSI_MAXQ + 1];
  std::unique_ptr<RnsArgs> sub_args[PEPSI_MAXQ + 1];
  // profiling
  bool prof = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<cudaEvent_t> ev_pool;
  uint64_t prof_launch[pepsi_detail::PC_COUNT] = {};
  double prof_ms[pepsi_detail::PC_COUNT] = {};
  uint64_t launches = 0;
};

namespace pepsi_detail {

// slots of d_consts
enum ConstSlot { CS_M3, CS_M7, CS_P12, CS_P16, CS_ZINV, CS_D_TM1, CS_D_2, CS_D_60, CS_COUNT };

// CK: in functions returning cudaError_t; CKS: in functions returning a PEPSI status
#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)
#define CKS(x)                                  \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

extern thread_local std::string g_last_error;
extern thread_local std::string g_detail;  // names the failing step for the next error report

int cuda_status(cudaError_t e);
bool is_device_ptr(const void* p);
cudaStream_t pick(pepsi_ctx* c, void* s);
// Layers per circuit chunk for n layers under the schedule's chunk: the
// fewest chunks of at most `chunk` layers, made as equal as possible (526
// layers at chunk 256: three chunks of 176 and 174 layers, not 256, 256, 14).
inline int balanced_chunk(int chunk, unsigned n) {
  if (n == 0) return 1;
  const unsigned want = (unsigned)std::max(1, chunk) < n ? (unsigned)std::max(1, chunk) : n;
  const unsigned parts = (n + want - 1) / want;
  return (int)((n + parts - 1) / parts);
}
// scratch slot `id` of the context with at least `bytes`
void* scratch(pepsi_ctx* c, int id, size_t bytes, cudaError_t* err);
void scratch_release(pepsi_ctx* c, int id);
void prof_collect(pepsi_ctx* c);

// Per-launch accounting (launch counts always; CUDA events when profiling).
struct Prof {
  pepsi_ctx* c;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(pepsi_ctx* c_, int cls_, cudaStream_t st_, int kernels = 1) : c(c_), cls(cls_), st(st_) {
    c->launches += kernels;
    c->prof_launch[cls] += kernels;
    if (!c->prof) return;
    if (c->ev_pool.size() < 2) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
      }
    }
    a = c->ev_pool.back();
    c->ev_pool.pop_back();
    b = c->ev_pool.back();
    c->ev_pool.pop_back();
    cudaEventRecord(a, st);
  }
  ~Prof() {
    if (!a) return;
    cudaEventRecord(b, st);
    c->prof_ev.push_back({cls, {a, b}});
  }
};

// Scratch layout of the evaluation pipeline for chunks of up to Lc layers.
struct EvalBufs {
  u64 *C, *H, *Hc, *XB, *YB, *T3, *D, *R, *U, *W, *X, *Y, *side, *acc, *Pc, *out, *zero;
};
enum ScratchId { S_C, S_H, S_HC, S_XB, S_YB, S_T3, S_D, S_R, S_U, S_W, S_X, S_Y, S_SIDE, S_ACC, S_PC, S_OUT, S_ZERO,
                 S_IN, S_DEC_Z, S_DEC_M, S_DEC_SLOTS, S_DEC_MAX, S_CT, S_POS, S_TC, S_HALL, S_COUNT };
cudaError_t eval_bufs(pepsi_ctx* c, int Lc, bool need_pc, EvalBufs* b);

// Operands of the last ciphertext product of the equality circuit, for L
// layers: Q parts in NTT form, B parts in NTT form, the constant added to
// the second operand's component 0 (Q residues, and its B extension per
// layer in `side`), and whether both operands are the same.
struct LastMult {
  const u64 *AQ = nullptr, *AB = nullptr, *BQ = nullptr, *BB = nullptr, *cQ = nullptr, *side = nullptr;
  bool square = false;
  // the same operands from layer `l` of the chunk on
  LastMult at(const pepsi_ctx* c, int l) const {
    const size_t qs = (size_t)l * 2 * c->k * c->N, bs = (size_t)l * 2 * c->kb * c->N;
    LastMult m = *this;
    m.AQ += qs;
    m.AB += bs;
    m.BQ += qs;
    m.BB += bs;
    if (m.side) m.side += (size_t)l * c->kb;
    return m;
  }
};

// Lazy rescaling state of one request: runs of G layers (counted from the
// first evaluated layer) share one rounding.  X holds the running sum of
// the run's exact products (NTT form over Q u B), acc the mod-Q layer sum.
struct LazyRun {
  u64* X;
  u64* acc;
  u32 G;
  u32 pos = 0;           // layers consumed so far
  bool acc_init = true;  // acc not yet written
};

// NTT rows [outer][np][N] with prime offset p0.
void ntt(pepsi_ctx* c, bool fwd, const u64* src, u64* dst, size_t outer, int np, int p0, size_t sos, size_t dos,
         cudaStream_t st);
// Arith-CW-Eq (Algorithm 1) on L layers whose h' is in b.H, up to its last
// ciphertext product (returned); and the whole circuit with per-layer rounding.
LastMult eq_circuit_front(pepsi_ctx* c, EvalBufs& b, int L, cudaStream_t st);
void eq_circuit(pepsi_ctx* c, EvalBufs& b, int L, cudaStream_t st);
// Lazy rescaling: add the chunk's last products to the run sums, rounding runs as they complete.
void lazy_chunk(pepsi_ctx* c, EvalBufs& b, const LastMult& m, const u64* VP, int L, bool end, LazyRun& r,
                cudaStream_t st);
// Run length of the lazy rescaling for an evaluation of nl layers in `mode`.
u32 rescale_run(const pepsi_ctx* c, u32 nl, int mode);
// Read and clear the device error flag (the stream must be synchronised).
bool take_error_flag(pepsi_ctx* c);
cudaError_t mac_status(cudaError_t e);
cudaError_t copy_any(void* dst, const void* src, size_t bytes, cudaStream_t st);
// a4: request ciphertexts (host or device) to NTT form in the split operand format, into C.
cudaError_t prepare_request(pepsi_ctx* c, const u64* cts, u64* C, cudaStream_t st);
// a7: relinearise the layer sum, times (h!)^-1, inverse NTT, mask, response switch, copy to out.
cudaError_t finish_request(pepsi_ctx* c, EvalBufs& b, u64* acc, bool acc_ntt, int mode, u64 mask_seed, u64* out,
                           cudaStream_t st);
// A context sharing the parent's keys, tables and server sets (device and
// host), with its own streams, events, error word and scratch: an
// evaluation lane.  Release it with pepsi_destroy, before the parent.
pepsi_ctx* ctx_fork(const pepsi_ctx* parent, cudaError_t* err);

}  // namespace pepsi_detail
