// Kernels of PEPSI's server evaluation (Algorithms 1, 2, 5) and the client
// steps around it (Algorithms 3, 7), for sm_103a.  Integer work only: the
// ciphertext arithmetic is 64-bit modular arithmetic on the CUDA cores.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "kernels.h"
#include "ntt_block.cuh"

namespace {

// Threads of a block running the register-blocked NTT: one per group of 8
// elements, at most 512 (two blocks of 64 KB per SM up to N = 8192), and
// 1024 at N = 16384, whose 128 KB polynomial leaves room for one block per
// SM.  The kernels below are compiled for 1024 threads at 64 registers, so
// either shape keeps 32 warps on an SM.
constexpr int NTT_MAX_THREADS = 1024;
inline int ntt_threads(int N) {
  if (N >= 16384) return NTT_MAX_THREADS;
  int t = N / 8;
  if (t > 512) t = 512;
  if (t < 32) t = 32;
  return t;
}
// Threads of the hot-path transform kernels: the schedule's choice
// (DevView::nt, picked by the autotuner), else the default above.
inline int xform_threads(const DevView& V) { return V.nt > 0 ? V.nt : ntt_threads(V.N); }
// SMs of the current device (cached per device).
inline int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!cached[dev]) cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev);
  return cached[dev];
}
// Threads of a transform launch of `rows` blocks: a launch that gives each
// block an SM of its own (the output stage, the lazy rounding) runs its
// rows with up to the largest blocks instead, which shortens each
// transform's chain of phases.
inline int xform_threads(const DevView& V, size_t rows) {
  const int base = xform_threads(V);
  const int wide = std::min(NTT_MAX_THREADS, std::max(32, V.N / 8));
  return rows <= (size_t)sm_count() && wide > base ? wide : base;
}
// The relinearisation transforms come in two register budgets: MT = 256 for
// blocks of at most 256 threads, three per SM (80 registers a thread; at N =
// 8192 with 256-thread blocks the relinearisation took 1.98 ms against
// 2.07 ms at 64), and MT = NTT_MAX_THREADS for larger blocks (64 registers).
constexpr int relin_min_blocks(int MT) { return MT <= 256 ? 3 : 1; }

// ------------------------------------------------------------------ NTT
// SPLIT: store the result in the split operand format of the
// multiply-accumulate (the request's forward transform).
template <bool FWD, bool SPLIT = false>
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_ntt(DevView V, const u64* __restrict__ src, u64* dst, int np, int p0, size_t src_os,
                      size_t dst_os, u32* sums) {
  extern __shared__ u64 sm[];
  const int N = V.N;
  const size_t r = blockIdx.x;
  const int pl = (int)(r % np);
  const size_t o = r / np;
  const u64* s = src + o * src_os + (size_t)pl * N;
  u64* d = dst + o * dst_os + (size_t)pl * N;
  const RowLd ld(s);
  if (FWD) {
    if (SPLIT)
      ntt_fwd_gg(sm, ld, SplitSumSt(d, sums + o * dst_os + (size_t)pl * N, V.pr[p0 + pl].split), V, p0 + pl);
    else
      ntt_fwd_gg(sm, ld, RowSt(d), V, p0 + pl);
  } else {
    ntt_inv_gg(sm, ld, RowSt(d), V, p0 + pl);
  }
}

// ------------------------------------------------ parallel cuckoo rounds
// One round of the client's cuckoo placement (pepsi_params.client_cuckoo =
// 1).  state: 0 placed, 1 unplaced, 2 evicted in this round; choice: the
// item's current candidate (0..2) among bins3[3u..3u+2].  claim[b] holds the
// smallest unplaced item claiming bin b (UINT32_MAX for none).
__global__ void k_ck_claim(const u32* __restrict__ bins3, const uint8_t* __restrict__ state,
                           const uint8_t* __restrict__ choice, u32 m, u32* claim) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= m || state[u] != 1) return;
  atomicMin(&claim[bins3[3 * (size_t)u + choice[u]]], u);
}
// Per bin: its winning claimant takes the first free slot, or the slot
// (evictions mod gamma) whose occupant is evicted to its next candidate.
__global__ void k_ck_resolve(u32 nbins, u32 gamma, u32* claim, int32_t* slot_item, u32* load, u32* evictions,
                             uint8_t* state, uint8_t* choice) {
  const u32 b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const u32 w = claim[b];
  if (w == 0xFFFFFFFFu) return;
  claim[b] = 0xFFFFFFFFu;
  size_t c;
  if (load[b] < gamma) {
    c = (size_t)b * gamma + load[b]++;
  } else {
    c = (size_t)b * gamma + evictions[b]++ % gamma;
    const int32_t v = slot_item[c];
    state[v] = 2;
    choice[v] = (uint8_t)((choice[v] + 1) % 3);
  }
  slot_item[c] = (int32_t)w;
  state[w] = 0;
}
// Claimants that lost move to their next candidate; the evicted become
// unplaced; *unplaced counts both.
__global__ void k_ck_advance(u32 m, uint8_t* state, uint8_t* choice, u32* unplaced) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= m) return;
  if (state[u] == 1) {
    choice[u] = (uint8_t)((choice[u] + 1) % 3);
    atomicAdd(unplaced, 1u);
  } else if (state[u] == 2) {
    state[u] = 1;
    atomicAdd(unplaced, 1u);
  }
}

// ---------------------------------------------------------- CW unranking
// v = sum_{r=1..h} C(c_r, r) with c_1 < ... < c_h (combinatorial number
// system); binom[c*(h+1)+r] = C(c, r) for c <= ell.
__global__ void k_cw_unrank(const u64* __restrict__ T, size_t count, const u64* __restrict__ binom, int ell, int h,
                            uint16_t* pos) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  u64 v = T[i];
  uint16_t* o = pos + i * h;
  if (v == PEPSI_DUMMY) {
    o[0] = PEPSI_CW_NONE;
    return;
  }
  int hi = ell;  // exclusive upper bound for c_r
  for (int r = h; r >= 1; --r) {
    // largest c in [r-1, hi) with C(c, r) <= v
    int lo = r - 1, up = hi - 1;
    while (lo < up) {
      int mid = (lo + up + 1) >> 1;
      if (binom[(size_t)mid * (h + 1) + r] <= v)
        lo = mid;
      else
        up = mid - 1;
    }
    o[r - 1] = (uint16_t)lo;
    v -= binom[(size_t)lo * (h + 1) + r];
    hi = lo;
  }
}

// ------------------------------------------------- server plaintexts (K3)
// Block (layer l, j-chunk): bit planes of the layer's codewords, encoded
// (inverse NTT mod t of the slot vector in bit-reversed order), centred
// lift into each q_p and forward NTT; stored in the split operand format.
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_ptgen(DevView V, const uint16_t* __restrict__ pos, int ell, int h, int JC, u64* P) {
  extern __shared__ u64 sm[];
  const int N = V.N, k = V.k;
  const int words = N / 32 > 0 ? N / 32 : 1;
  u64* poly = sm;                                  // N u64
  u32* mbuf = reinterpret_cast<u32*>(sm + N);      // N u32
  u32* bits = mbuf + N;                            // JC * words u32
  const int l = blockIdx.y;
  const int j0 = blockIdx.x * JC;
  for (int x = threadIdx.x; x < JC * words; x += blockDim.x) bits[x] = 0;
  __syncthreads();
  const uint16_t* lp = pos + (size_t)l * N * h;
  for (int s = threadIdx.x; s < N; s += blockDim.x) {
    const uint16_t* ps = lp + (size_t)s * h;
    if (ps[0] == PEPSI_CW_NONE) continue;
    for (int r = 0; r < h; ++r) {
      int c = (int)ps[r] - j0;
      if (c >= 0 && c < JC) atomicOr(&bits[c * words + (s >> 5)], 1u << (s & 31));
    }
  }
  __syncthreads();
  const DevPrime Pt = V.pr[V.tidx];
  const u64 t = Pt.q, thalf = t >> 1;
  for (int jj = 0; jj < JC; ++jj) {
    const int j = j0 + jj;
    if (j >= ell) break;
    // Encode: slot s at position brev(s), inverse NTT mod t into mbuf (in
    // 32-bit words for t below 2^30)
    const u32* bj = bits + jj * words;
    if (t < (1ull << 30)) {
      ntt_inv_gg_small(
          reinterpret_cast<u32*>(poly),
          [&](int i) -> u32 {
            const u32 s = brev_bits(i, V.logN);
            return (bj[s >> 5] >> (s & 31)) & 1u;
          },
          [&](int i, u32 v) { mbuf[i] = v; }, V, V.tidx);
    } else {
      ntt_inv_gg(
          poly,
          [&](int i) -> u64 {
            const u32 s = brev_bits(i, V.logN);
            return (bj[s >> 5] >> (s & 31)) & 1u;
          },
          [&](int i, u64 v) { mbuf[i] = (u32)v; }, V, V.tidx);
    }
    __syncthreads();
    for (int p = 0; p < k; ++p) {
      // centred lift to q_p on the load, split operand format on the store
      const u64 q = V.pr[p].q, sp = V.pr[p].split;
      u64* out = P + (((size_t)l * ell + j) * k + p) * N;
      ntt_fwd_gg(
          poly,
          [&](int i) -> u64 {
            const u64 m = mbuf[i];
            return m <= thalf ? m : q - (t - m);
          },
          SplitSt(out, sp), V, p);
      __syncthreads();  // the next transform overwrites poly
    }
  }
}

// Value plaintexts of labelled PSI / PSI-Sum (Algorithms 4-5): for layer
// l (one block each), slots V[l][.] -> Encode (inverse NTT mod t, slot s at
// position brev(s)) -> centred lift -> forward NTT for every prime of
// Q u B.  Out VP[l][k+kb][N] (plain residues, not the split format).
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_valgen(DevView V, const u32* __restrict__ vals, u64* VP) {
  extern __shared__ u64 sm[];
  const int N = V.N, np = V.k + V.kb;
  u64* poly = sm;                              // N u64
  u32* mbuf = reinterpret_cast<u32*>(sm + N);  // N u32
  const int l = blockIdx.x;
  const u32* row = vals + (size_t)l * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) poly[nsw(i)] = row[brev_bits(i, V.logN)];
  __syncthreads();
  ntt_inv_view(poly, V, V.tidx);
  for (int i = threadIdx.x; i < N; i += blockDim.x) mbuf[i] = (u32)poly[nsw(i)];
  __syncthreads();
  const u64 t = V.pr[V.tidx].q, thalf = t >> 1;
  for (int p = 0; p < np; ++p) {
    const u64 q = V.pr[p].q;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const u64 m = mbuf[i];
      poly[nsw(i)] = m <= thalf ? m : q - (t - m);
    }
    __syncthreads();
    ntt_fwd_view(poly, V, p);
    u64* out = VP + ((size_t)l * np + p) * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) out[i] = poly[nsw(i)];
    __syncthreads();
  }
}

// ------------------------------------------------------- fused MAC (K4)
// h'[l] = sum_j C[j] * P[l][j] pointwise in the NTT domain, for both
// ciphertext components.  A block owns TN consecutive (prime, point) words
// and LB layers.  One producer thread streams P and C tiles of JS codeword
// bits through NST shared-memory stages, each stage two tiled TMA copies
// (cp.async.bulk.tensor.3d: a TN x JS x LB box of P and a TN x 2 x JS box of
// C, completion counted on a "full" mbarrier); consumer warps release a
// stage through an "empty" mbarrier.  Boxes that cross the end of a
// dimension are zero-filled by the copy engine, and zeros add nothing.
// Each consumer thread owns one point and LPT layers.  Operands are in the
// split format (x = hi 2^s + lo, both halves below 2^32): a 64-bit product
// is three 32x32->64 multiply-adds in Karatsuba form into three 64-bit
// partial sums, folded into the reduced accumulator before they can
// overflow.  The plaintext tile may also come as 7-byte words in three
// planes (P7), put back together on the load.  Every mbarrier
// wait is bounded (about one second); on expiry the block waits, again
// bounded, for its own copies in flight, sets *err and returns.
// Five 44 KB stages (220 KB of the 227 KB a block may hold): at the paper
// shape a fifth stage took the launch from 12.13 to 11.94 ms, while stages
// of 2, 3, 5 or 6 bits, or 16 layers a block, were no faster.
namespace mac {
constexpr int TN = 128, LB = 8, LPT = 2, JS = 4, NST = 5;
constexpr int LG = LB / LPT;                    // layer slices per block
constexpr int CONSUMER_WARPS = (TN / 32) * LG;  // 16
constexpr int THREADS = (CONSUMER_WARPS + 1) * 32;
constexpr int P_WORDS = LB * JS * TN, C_WORDS = 2 * JS * TN;
// A stage holds the plaintext tile, then the request tile and the request's
// half sums (4 bytes per word, read instead of added by every layer slice).
// The plaintext tile is 8 bytes per word (split operand format), or 7 bytes
// per word in three planes one after another: bits 0-31, 32-47 and 48-55 of
// the value.
template <bool P7>
__host__ __device__ constexpr int p_bytes() {
  return P_WORDS * (P7 ? 7 : 8);
}
template <bool P7>
__host__ __device__ constexpr int stage_bytes() {
  return p_bytes<P7>() + C_WORDS * 12;
}
template <bool P7>
__host__ __device__ constexpr size_t smem() {
  return (size_t)NST * stage_bytes<P7>() + 2 * NST * 8 + 16 + 128;
}
}  // namespace mac

__device__ __forceinline__ u64 globaltimer_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(u32 addr, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u32 addr, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(u32 addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u32 addr, u32 parity) {
  u32 ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of an mbarrier for at most about one second.
__device__ __forceinline__ bool mbar_wait_bounded(u32 addr, u32 parity) {
  if (mbar_try_wait(addr, parity)) return true;
  const u64 t0 = globaltimer_ns();
  while (!mbar_try_wait(addr, parity))
    if (globaltimer_ns() - t0 > 1000000000ull) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(u32 dst, const CUtensorMap* tm, int c0, int c1, int c2, u32 bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<u64>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
// acc += a * b for 32-bit a, b into a 64-bit sum (one wide multiply-add).
// Measured on this GPU with operands that change every step: 7.0 T such
// accumulations per second (the product alone, mul.wide.u32, 18 T/s).  A
// carry-chained pair of 32-bit multiply-adds (9.5 T/s in isolation) and a
// product plus separate 64-bit adds gave no faster multiply-accumulate.
__device__ __forceinline__ void mad_wide(u64& acc, u32 a, u32 b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}
// The first 128-byte boundary of the dynamic shared memory, as an offset
// from the array itself (the compiler then keeps the shared address space).
__device__ __forceinline__ unsigned char* stage_base(u64* raw) {
  const u32 a = (u32)__cvta_generic_to_shared(raw);
  return reinterpret_cast<unsigned char*>(raw) + ((128u - (a & 127u)) & 127u);
}
// Karatsuba form of a split product c x = (ch 2^s + cl)(xh 2^s + xl): three
// wide multiply-adds, S0 += cl xl, S2 += ch xh, SM += (cl + ch)(xl + xh),
// instead of four.  The middle sum S1 = sum cl xh + ch xl is SM - S0 - S2
// at the fold, exact mod 2^64: SM may wrap, S0, S1 and S2 stay below 2^64.
// (Taking S2 and SM as a product plus a separate 64-bit add, which moves
// work from the multiply-add pipe to the ALU and runs twice as fast in
// isolation, left both multiply-accumulate kernels within 3% of this form.)
__device__ __forceinline__ void kmac(u64& S0, u64& SM, u64& S2, u32 cl, u32 ch, u32 cs, u32 xl, u32 xh, u32 xs) {
  mad_wide(S0, cl, xl);
  mad_wide(S2, ch, xh);
  mad_wide(SM, cs, xs);
}
// S0 + (SM - S0 - S2) 2^s + S2 2^2s as a 128-bit value (hi, lo)
__device__ __forceinline__ void compose(u64 S0, u64 SM, u64 S2, u64 s, u64& hi, u64& lo) {
  const u64 S1 = SM - S0 - S2;
  lo = S0;
  hi = 0;
  const u64 a = S1 << s;
  hi += S1 >> (64 - s);
  lo += a;
  hi += lo < a;
  const u64 b = S2 << (2 * s);
  hi += S2 >> (64 - 2 * s);
  lo += b;
  hi += lo < b;
}
// The sums reduced mod q back into S0 and SM (S2 = 0): both restart at the
// residue r, so SM - S0 stays the middle term; the fold interval leaves
// room for r below 2^64.
__device__ __forceinline__ void fold_inplace(u64& S0, u64& SM, u64& S2, u64 s, const DevPrime& pr) {
  u64 hi, lo;
  compose(S0, SM, S2, s, hi, lo);
  S0 = SM = reduce128(hi, lo, pr);
  S2 = 0;
}
__device__ __forceinline__ void fold_into(u64& acc, u64& S0, u64& SM, u64& S2, u64 s, const DevPrime& pr) {
  u64 hi, lo;
  compose(S0, SM, S2, s, hi, lo);
  acc = addmod(acc, reduce128(hi, lo, pr), pr.q);
  S0 = SM = S2 = 0;
}

// Plaintext word o of a stage's tile as split operands xl = x mod 2^s,
// xh = x >> s.  P7: x is put together from its three planes.
template <bool P7>
__device__ __forceinline__ void tile_word(const unsigned char* stg, int o, u32 s, u32 lmask, u32& xl, u32& xh) {
  if constexpr (P7) {
    const u32 a = reinterpret_cast<const u32*>(stg)[o];
    const u32 b = reinterpret_cast<const uint16_t*>(stg + mac::P_WORDS * 4)[o];
    const u32 c = stg[mac::P_WORDS * 6 + o];
    const u32 hi = __byte_perm(b, c, 0x2410);  // b | c << 16: bits 32-55 of x
    xl = a & lmask;
    xh = __funnelshift_r(a, hi, s);
  } else {
    const u64 x = reinterpret_cast<const u64*>(stg)[o];
    xl = (u32)x;
    xh = (u32)(x >> 32);
  }
}
// The stage's plaintext copies: one tensor copy of the words, or one per plane.
template <bool P7>
__device__ __forceinline__ void tma_plain(u32 sb, const CUtensorMap* tmP, const CUtensorMap* tmPb,
                                          const CUtensorMap* tmPc, int x, int j, int l, u32 bar) {
  tma_load_3d(sb, tmP, x, j, l, bar);
  if constexpr (P7) {
    tma_load_3d(sb + mac::P_WORDS * 4, tmPb, x, j, l, bar);
    tma_load_3d(sb + mac::P_WORDS * 6, tmPc, x, j, l, bar);
  }
}

// One launch covers the codeword bits [j0, j0 + nj) (nj a multiple of JS
// unless the range ends at ell); with acc_in it adds to the h' already in
// H, so a request can be multiplied in pieces as it arrives.
template <bool P7>
__global__ void __launch_bounds__(mac::THREADS, 1)
    k_mac(DevView V, const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmPb,
          const __grid_constant__ CUtensorMap tmPc, const __grid_constant__ CUtensorMap tmC,
          const __grid_constant__ CUtensorMap tmS, u64* __restrict__ H, int j0, int nj, int L, int fold_stages,
          int acc_in, int* err) {
  using namespace mac;
  constexpr int SB = stage_bytes<P7>(), PB = p_bytes<P7>();
  extern __shared__ __align__(128) u64 sm_raw[];
  // 128-byte aligned stage buffers for the tensor copies, derived from the
  // shared array by pointer arithmetic so that its loads stay shared-memory
  // loads
  unsigned char* sm = stage_base(sm_raw);
  const size_t kN = (size_t)V.k * V.N;
  const int l0 = blockIdx.x * LB;
  const int nl = min(LB, L - l0);
  const size_t idx0 = (size_t)blockIdx.y * TN;
  const int cnt = (int)min((size_t)TN, kN - idx0);
  const int nst = (nj + JS - 1) / JS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 sbase = (u32)__cvta_generic_to_shared(sm);
  const u32 full0 = sbase + (u32)(NST * SB), empty0 = full0 + NST * 8;
  int* abort_flag = reinterpret_cast<int*>(sm + NST * SB + 2 * NST * 8);
  if (threadIdx.x == 0) {
    for (int b = 0; b < NST; ++b) {
      mbar_init(full0 + 8 * b, 1);
      mbar_init(empty0 + 8 * b, CONSUMER_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = true;
  int issued = 0;  // producer: stages issued
  if (warp == CONSUMER_WARPS) {
    // ---------------- producer: one thread issues the tensor copies of each stage
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&tmP)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&tmC)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&tmS)) : "memory");
      for (int st = 0; st < nst; ++st) {
        const int buf = st % NST;
        if (st >= NST && !mbar_wait_bounded(empty0 + 8 * buf, (u32)(((st / NST) - 1) & 1))) {
          ok = false;
          break;
        }
        const u32 bar = full0 + 8 * buf;
        const u32 sb = sbase + (u32)(buf * SB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (u32)SB);
        tma_plain<P7>(sb, &tmP, &tmPb, &tmPc, (int)idx0, j0 + st * JS, l0, bar);
        tma_load_3d(sb + (u32)PB, &tmC, (int)idx0, 0, j0 + st * JS, bar);
        tma_load_3d(sb + (u32)(PB + C_WORDS * 8), &tmS, (int)idx0, 0, j0 + st * JS, bar);
        issued = st + 1;
      }
    }
  } else {
    // ---------------- consumer warps
    const int tp = (warp % (TN / 32)) * 32 + lane;  // point within the tile
    const int g = warp / (TN / 32);                 // layer slice
    const bool active = tp < cnt;
    const size_t idx = idx0 + (active ? tp : 0);
    const DevPrime pr = V.pr[idx / V.N];
    const u64 sp = pr.split;
    const u32 s32 = (u32)sp, lmask = (1u << s32) - 1;
    u64 S0[LPT][2], SM[LPT][2], S2[LPT][2], acc[LPT][2];
#pragma unroll
    for (int l = 0; l < LPT; ++l)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        S0[l][c] = SM[l][c] = S2[l][c] = acc[l][c] = 0;
        const int layer = g * LPT + l;
        if (acc_in && active && layer < nl) acc[l][c] = H[((size_t)(l0 + layer) * 2 + c) * kN + idx];
      }
    int since = 0;
    for (int st = 0; st < nst; ++st) {
      const int buf = st % NST;
      if (!mbar_wait_bounded(full0 + 8 * buf, (u32)((st / NST) & 1))) {
        ok = false;
        break;
      }
      const unsigned char* stg = sm + (size_t)buf * SB;
      const int po = g * LPT * JS * TN + tp;  // word (slice, bit 0, point) of the tile
      const u64* cs = reinterpret_cast<const u64*>(stg + PB) + tp;
      const u32* ss = reinterpret_cast<const u32*>(stg + PB + C_WORDS * 8) + tp;
#pragma unroll
      for (int jj = 0; jj < JS; ++jj) {
        const u64 c0 = cs[(jj * 2) * TN], c1 = cs[(jj * 2 + 1) * TN];
        const u32 c0l = (u32)c0, c0h = (u32)(c0 >> 32), c1l = (u32)c1, c1h = (u32)(c1 >> 32);
        const u32 c0s = ss[(jj * 2) * TN], c1s = ss[(jj * 2 + 1) * TN];
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
          u32 xl, xh;
          tile_word<P7>(stg, po + (l * JS + jj) * TN, s32, lmask, xl, xh);
          const u32 xs = xl + xh;
          kmac(S0[l][0], SM[l][0], S2[l][0], c0l, c0h, c0s, xl, xh, xs);
          kmac(S0[l][1], SM[l][1], S2[l][1], c1l, c1h, c1s, xl, xh, xs);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * buf);
      if (++since == fold_stages) {
#pragma unroll
        for (int l = 0; l < LPT; ++l)
#pragma unroll
          for (int c = 0; c < 2; ++c) fold_into(acc[l][c], S0[l][c], SM[l][c], S2[l][c], sp, pr);
        since = 0;
      }
    }
    if (ok && active) {
#pragma unroll
      for (int l = 0; l < LPT; ++l)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          fold_into(acc[l][c], S0[l][c], SM[l][c], S2[l][c], sp, pr);
          const int layer = g * LPT + l;
          if (layer < nl) H[((size_t)(l0 + layer) * 2 + c) * kN + idx] = acc[l][c];
        }
    }
  }
  if (!ok) atomicExch(abort_flag, 1);
  __syncthreads();
  if (*abort_flag && warp == CONSUMER_WARPS && lane == 0) {
    // copies of the last NST issued stages may still be landing: wait for them
    for (int st = max(0, issued - NST); st < issued; ++st)
      mbar_wait_bounded(full0 + 8 * (st % NST), (u32)((st / NST) & 1));
    atomicExch(err, 1);
  }
}

// Multi-request variant: QB <= 4 requests against the same plaintexts.
// Each plaintext tile is read from HBM once and feeds 2*QB products per
// word, so the batch's plaintext stream costs what one request's does and
// the kernel is bound by the wide multiply-adds instead (6 per plaintext
// word and request).  A block owns TN = 32*WPS consecutive (prime, point)
// words and LB = 16/WPS layers.  Each of the 8 consumer warps covers 32
// points of one layer slice; each consumer thread one point, LPT = 2 layers
// and all QB requests: a plaintext word loaded from shared memory serves
// 2*QB products and a request word (with its half sum) LPT products, so a
// 4-request batch reads 10 shared-memory words and 8 half sums per 48
// multiply-adds (the SM's shared-memory bandwidth is a quarter of its wide
// multiply-add rate in 8-byte words).
// Its 48 64-bit partial sums per thread are why there are 8 consumer warps:
// with the producer, 9 warps put at most 3 on an SM sub-partition, whose
// 16K registers then allow 168 per thread (13 warps would cap them at
// 128 and spill).  Each request's tile is two 3-D TMA boxes (points x
// components x bits: its split words and their half sums, plain loads of
// this GPU's memory).  Same
// pipeline, split operands, Karatsuba sums, folding and bounded waits as
// k_mac.  Each request has its own tensor map and output, so the requests
// may live anywhere; the tile width WPS is a schedule choice (wider rows per copy
// against fewer re-reads of the request tiles, which every layer group
// reads again from L2).
namespace macq {
constexpr int LPT = 2, JS = 4, NST = 4, QMAX = 4, GROUP_WARPS = 8;
static_assert(QMAX == PEPSI_MAC_MAX_REQUESTS, "one request bound");
// RG request groups of GROUP_WARPS consumer warps each, plus the producer warp
__host__ __device__ constexpr int threads(int RG) { return (GROUP_WARPS * RG + 1) * 32; }
template <int WPS>
struct Tile {
  static constexpr int TN = 32 * WPS;                // points per block
  static constexpr int LG = GROUP_WARPS / WPS;       // layer slices
  static constexpr int LB = LG * LPT;                // layers per block
  static constexpr int P_WORDS = LB * JS * TN;
  static_assert(LG * WPS == GROUP_WARPS, "whole layer slices");
};
template <int QB, int WPS, bool P7>
__host__ __device__ constexpr int p_bytes() {
  return Tile<WPS>::P_WORDS * (P7 ? 7 : 8);
}
// request q's tile of split words, then its tile of half sums
template <int WPS>
__host__ __device__ constexpr int req_bytes() {
  return 2 * JS * Tile<WPS>::TN * 12;
}
template <int QB, int WPS, bool P7>
__host__ __device__ constexpr int stage_bytes() {
  return p_bytes<QB, WPS, P7>() + QB * req_bytes<WPS>();
}
template <int QB, int WPS, bool P7>
__host__ __device__ constexpr size_t smem() {
  return (size_t)NST * stage_bytes<QB, WPS, P7>() + 2 * NST * 8 + 16 + 128;
}
}  // namespace macq

__device__ __forceinline__ void tma_load_4d(u32 dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3, u32 bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<u64>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Plaintext word o of a stage tile of PW words (see tile_word), and the
// stage's plaintext copies for that tile size.
template <bool P7, int PW>
__device__ __forceinline__ void tile_word_pw(const unsigned char* stg, int o, u32 s, u32 lmask, u32& xl, u32& xh) {
  if constexpr (P7) {
    const u32 a = reinterpret_cast<const u32*>(stg)[o];
    const u32 b = reinterpret_cast<const uint16_t*>(stg + PW * 4)[o];
    const u32 c = stg[PW * 6 + o];
    const u32 hi = __byte_perm(b, c, 0x2410);
    xl = a & lmask;
    xh = __funnelshift_r(a, hi, s);
  } else {
    const u64 x = reinterpret_cast<const u64*>(stg)[o];
    xl = (u32)x;
    xh = (u32)(x >> 32);
  }
}
template <bool P7, int PW>
__device__ __forceinline__ void tma_plain_pw(u32 sb, const CUtensorMap* tmP, const CUtensorMap* tmPb,
                                             const CUtensorMap* tmPc, int x, int j, int l, u32 bar) {
  tma_load_3d(sb, tmP, x, j, l, bar);
  if constexpr (P7) {
    tma_load_3d(sb + PW * 4, tmPb, x, j, l, bar);
    tma_load_3d(sb + PW * 6, tmPc, x, j, l, bar);
  }
}

template <int QB, int RG, int WPS, bool P7>
__global__ void __launch_bounds__(macq::threads(RG), 1)
    k_mac_multi(DevView V, const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmPb,
                const __grid_constant__ CUtensorMap tmPc, const __grid_constant__ MacRequests rq, int ell, int L,
                int fold_stages, int* err) {
  using namespace macq;
  using TL = Tile<WPS>;
  constexpr int CONSUMER_WARPS = GROUP_WARPS * RG, QT = QB / RG;  // QT requests per consumer thread
  static_assert(QT * RG == QB, "whole request groups");
  constexpr int TN = TL::TN, LB = TL::LB, PW = TL::P_WORDS;
  constexpr int SB = stage_bytes<QB, WPS, P7>(), PB = p_bytes<QB, WPS, P7>();
  extern __shared__ __align__(128) u64 sm_raw[];
  unsigned char* sm = stage_base(sm_raw);
  const size_t kN = (size_t)V.k * V.N;
  const int l0 = blockIdx.x * LB;
  const int nl = min(LB, L - l0);
  const size_t idx0 = (size_t)blockIdx.y * TN;
  const int cnt = (int)min((size_t)TN, kN - idx0);
  const int nst = (ell + JS - 1) / JS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 sbase = (u32)__cvta_generic_to_shared(sm);
  const u32 full0 = sbase + (u32)(NST * SB), empty0 = full0 + NST * 8;
  int* abort_flag = reinterpret_cast<int*>(sm + NST * SB + 2 * NST * 8);
  if (threadIdx.x == 0) {
    for (int b = 0; b < NST; ++b) {
      mbar_init(full0 + 8 * b, 1);
      mbar_init(empty0 + 8 * b, CONSUMER_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = true;
  int issued = 0;
  if (warp == CONSUMER_WARPS) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&tmP)) : "memory");
#pragma unroll
      for (int q = 0; q < QB; ++q) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&rq.c[q])) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&rq.s[q])) : "memory");
      }
      for (int st = 0; st < nst; ++st) {
        const int buf = st % NST;
        if (st >= NST && !mbar_wait_bounded(empty0 + 8 * buf, (u32)(((st / NST) - 1) & 1))) {
          ok = false;
          break;
        }
        const u32 bar = full0 + 8 * buf;
        const u32 sb = sbase + (u32)(buf * SB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (u32)SB);
        tma_plain_pw<P7, PW>(sb, &tmP, &tmPb, &tmPc, (int)idx0, st * JS, l0, bar);
#pragma unroll
        for (int q = 0; q < QB; ++q) {
          const u32 rb = sb + (u32)(PB + q * req_bytes<WPS>());
          tma_load_3d(rb, &rq.c[q], (int)idx0, 0, st * JS, bar);
          tma_load_3d(rb + (u32)(2 * JS * TN * 8), &rq.s[q], (int)idx0, 0, st * JS, bar);
        }
        issued = st + 1;
      }
    }
  } else {
    const int rg = warp / GROUP_WARPS, gw = warp % GROUP_WARPS;  // request group, warp within it
    const int tp = (gw % WPS) * 32 + lane;  // point within the tile
    const int g = gw / WPS;                 // layer slice
    const bool active = tp < cnt;
    const size_t idx = idx0 + (active ? tp : 0);
    const DevPrime pr = V.pr[idx / V.N];
    const u64 sp = pr.split;
    const u32 s32 = (u32)sp, lmask = (1u << s32) - 1;
    u64 S0[LPT][QT][2], SM[LPT][QT][2], S2[LPT][QT][2];
#pragma unroll
    for (int l = 0; l < LPT; ++l)
#pragma unroll
      for (int q = 0; q < QT; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c) S0[l][q][c] = SM[l][q][c] = S2[l][q][c] = 0;
    int since = 0;
    for (int st = 0; st < nst; ++st) {
      const int buf = st % NST;
      if (!mbar_wait_bounded(full0 + 8 * buf, (u32)((st / NST) & 1))) {
        ok = false;
        break;
      }
      const unsigned char* stg = sm + (size_t)buf * SB;
      const int po = g * LPT * JS * TN + tp;  // word (slice, bit 0, point) of the plaintext tile
      const unsigned char* rqt = stg + PB + rg * QT * req_bytes<WPS>();  // this group's request tiles
#pragma unroll
      for (int jj = 0; jj < JS; ++jj) {
        u32 xl[LPT], xh[LPT], xs[LPT];
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
          tile_word_pw<P7, PW>(stg, po + (l * JS + jj) * TN, s32, lmask, xl[l], xh[l]);
          xs[l] = xl[l] + xh[l];
        }
#pragma unroll
        for (int q = 0; q < QT; ++q)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const unsigned char* t = rqt + q * req_bytes<WPS>();
            const u64 w = reinterpret_cast<const u64*>(t)[(jj * 2 + c) * TN + tp];
            const u32 cl = (u32)w, ch = (u32)(w >> 32);
            const u32 csum = reinterpret_cast<const u32*>(t + 2 * JS * TN * 8)[(jj * 2 + c) * TN + tp];
#pragma unroll
            for (int l = 0; l < LPT; ++l)
              kmac(S0[l][q][c], SM[l][q][c], S2[l][q][c], cl, ch, csum, xl[l], xh[l], xs[l]);
          }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * buf);
      if (++since == fold_stages) {
#pragma unroll
        for (int l = 0; l < LPT; ++l)
#pragma unroll
          for (int q = 0; q < QT; ++q)
#pragma unroll
            for (int c = 0; c < 2; ++c) fold_inplace(S0[l][q][c], SM[l][q][c], S2[l][q][c], sp, pr);
        since = 0;
      }
    }
    if (ok && active) {
#pragma unroll
      for (int l = 0; l < LPT; ++l)
#pragma unroll
        for (int q = 0; q < QT; ++q)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            fold_inplace(S0[l][q][c], SM[l][q][c], S2[l][q][c], sp, pr);
            const int layer = g * LPT + l;
            if (layer < nl) rq.h[rg * QT + q][((size_t)(l0 + layer) * 2 + c) * kN + idx] = S0[l][q][c];
          }
    }
  }
  if (!ok) atomicExch(abort_flag, 1);
  __syncthreads();
  if (*abort_flag && warp == CONSUMER_WARPS && lane == 0) {
    for (int st = max(0, issued - NST); st < issued; ++st)
      mbar_wait_bounded(full0 + 8 * (st % NST), (u32)((st / NST) & 1));
    atomicExch(err, 1);
  }
}

// In-place conversion of [rows][N] words between the reduced and the split
// operand format; row r uses prime r % k.
__global__ void k_split(DevView V, u64* x, size_t total, int to) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const u64 s = V.pr[(i / V.N) % V.k].split;
  x[i] = to ? to_split(x[i], s) : from_split(x[i], s);
}

// Split-format words of rows [..][k][N] (row r uses prime r % k) to the
// three planes of the 7-byte format: bits 0-31, 32-47 and 48-55 of each
// reduced value (every prime below 2^56).
__global__ void k_pack7(DevView V, const u64* __restrict__ src, size_t count, u32* a, uint16_t* b, uint8_t* c) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const u64 x = from_split(src[i], V.pr[(i / V.N) % V.k].split);
  a[i] = (u32)x;
  b[i] = (uint16_t)(x >> 32);
  c[i] = (uint8_t)(x >> 48);
}
// The reduced values back from the three planes.
__global__ void k_unpack7(const u32* __restrict__ a, const uint16_t* __restrict__ b, const uint8_t* __restrict__ c,
                          size_t count, u64* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  out[i] = (u64)a[i] | ((u64)b[i] << 32) | ((u64)c[i] << 48);
}

// ---------------------------------------------------- RNS conversions
// Templated on the numbers of Q and B primes (0: read them at run time) so
// that digit arrays stay in registers; primes and constants come by value
// in the kernel parameter space (RnsArgs).

// Garner mixed-radix digits v over Q of residues x.
template <int K>
__device__ __forceinline__ void garner_q(const RnsArgs& A, const u64* x, u64* v) {
  constexpr int M = K ? K : PEPSI_MAXQ;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    if (K || i < A.k) {
      const DevPrime pi = A.pr[i];
      u64 acc = x[i];
#pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j < i) {
          const u64 vj = v[j] >= pi.q ? barrett64(v[j], pi) : v[j];
          acc = submod(acc, vj, pi.q);
          acc = shoup(acc, A.rc.cq[i][j], A.rc.cqs[i][j], pi.q);
        }
      }
      v[i] = acc;
    }
  }
}
// Garner mixed-radix digits u over B of residues y.
template <int K, int KB>
__device__ __forceinline__ void garner_b(const RnsArgs& A, const u64* y, u64* u) {
  constexpr int M = KB ? KB : PEPSI_MAXB;
  const int k = K ? K : A.k;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    if (KB || i < A.kb) {
      const DevPrime pi = A.pr[k + i];
      u64 acc = y[i];
#pragma unroll
      for (int j = 0; j < M; ++j) {
        if (j < i) {
          const u64 uj = u[j] >= pi.q ? barrett64(u[j], pi) : u[j];
          acc = submod(acc, uj, pi.q);
          acc = shoup(acc, A.rc.cb[i][j], A.rc.cbs[i][j], pi.q);
        }
      }
      u[i] = acc;
    }
  }
}
// true when the mixed-radix number v (n digits, M at most) exceeds h
template <int M>
__device__ __forceinline__ bool digits_greater(const u64* v, const u64* h, int n) {
  bool gt = false, decided = false;
#pragma unroll
  for (int i = M - 1; i >= 0; --i) {
    if (i < n && !decided && v[i] != h[i]) {
      gt = v[i] > h[i];
      decided = true;
    }
  }
  return gt;
}
// value of the Q-digits v (centred when neg) reduced mod B prime j, by
// Horner's rule v_0 + q_0 (v_1 + q_1 (v_2 + ...)) with Shoup products: every
// partial value stays below 2 p_j + 2^60, one reduction at the end
template <int K>
__device__ __forceinline__ u64 q_digits_mod_b(const RnsArgs& A, const u64* v, bool neg, int j) {
  constexpr int M = K ? K : PEPSI_MAXQ;
  const int k = K ? K : A.k;
  const DevPrime pb = A.pr[k + j];
  u64 acc = v[k - 1];
#pragma unroll
  for (int l = M - 2; l >= 0; --l)
    if (K || l < k - 1) acc = shoup_lazy(acc, A.rc.qb[j][l], A.rc.qbs[j][l], pb.q) + v[l];
  const u64 r = barrett64(acc, pb);
  return neg ? submod(r, A.rc.qmodb[j], pb.q) : r;
}

template <int K, int KB>
__global__ void k_lift(const __grid_constant__ RnsArgs A, const u64* __restrict__ src, u64* __restrict__ dstB,
                       int L, const u64* __restrict__ cst, u64* __restrict__ side) {
  constexpr int MQ = K ? K : PEPSI_MAXQ, MB = KB ? KB : PEPSI_MAXB;
  const int N = A.N, k = K ? K : A.k, kb = KB ? KB : A.kb;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over L*2*N
  if (idx >= (size_t)L * 2 * N) return;
  const int n = (int)(idx % N);
  const size_t lc = idx / N;  // layer*2 + comp
  u64 x[MQ], v[MQ];
#pragma unroll
  for (int i = 0; i < MQ; ++i)
    if (K || i < k) x[i] = src[(lc * k + i) * N + n];
  garner_q<K>(A, x, v);
  const bool neg = digits_greater<MQ>(v, A.rc.qhalf_dig, k);
  u64 base[MB];
#pragma unroll
  for (int j = 0; j < MB; ++j)
    if (KB || j < kb) {
      base[j] = q_digits_mod_b<K>(A, v, neg, j);
      dstB[(lc * kb + j) * N + n] = base[j];
    }
  if (cst != nullptr && n == 0 && (lc & 1) == 0) {
    // lift of (x + cst) mod Q at coefficient 0 of component 0
#pragma unroll
    for (int i = 0; i < MQ; ++i)
      if (K || i < k) x[i] = addmod(x[i], cst[i], A.pr[i].q);
    garner_q<K>(A, x, v);
    const bool neg2 = digits_greater<MQ>(v, A.rc.qhalf_dig, k);
    const size_t layer = lc >> 1;
#pragma unroll
    for (int j = 0; j < MB; ++j)
      if (KB || j < kb) side[layer * kb + j] = submod(q_digits_mod_b<K>(A, v, neg2, j), base[j], A.pr[k + j].q);
  }
}

// ------------------------------------------------------------ tensor
// Tensor product fused with its inverse transform: block per row
// (l, c, pi) of T3[L][3][k+kb][N] computes component c of the tensor of
// (A_l, B_l) at prime pi on the load of the inverse NTT, and stores the
// coefficient-form row: the tensor (a0b0, a0b1 + a1b0, a1b1) and its
// inverse NTT without a round trip of the NTT-form tensor through memory.
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1)
    k_tensor_intt(DevView V, const u64* __restrict__ AQ, const u64* __restrict__ AB, const u64* __restrict__ BQ,
                  const u64* __restrict__ BB, const u64* __restrict__ cstQ, const u64* __restrict__ side,
                  u64* __restrict__ T3, int square) {
  extern __shared__ u64 sm[];
  const int N = V.N, k = V.k, kb = V.kb, np = k + kb;
  const size_t r = blockIdx.x;
  const int pi = (int)(r % np);
  const size_t o = r / np;  // l * 3 + c
  const int c = (int)(o % 3);
  const size_t l = o / 3;
  const DevPrime pr = V.pr[pi];
  const u64 *A, *Bp;
  size_t o0, o1;
  u64 cb = 0;  // constant added to b0 (NTT form: the same at every point)
  if (pi < k) {
    A = AQ;
    Bp = BQ;
    o0 = ((l * 2 + 0) * k + pi) * N;
    o1 = ((l * 2 + 1) * k + pi) * N;
    if (!square && cstQ) cb = cstQ[pi];
  } else {
    A = AB;
    Bp = BB;
    o0 = ((l * 2 + 0) * kb + (pi - k)) * N;
    o1 = ((l * 2 + 1) * kb + (pi - k)) * N;
    if (!square && side) cb = side[l * kb + (pi - k)];
  }
  const u64* a0 = A + o0;
  const u64* a1 = A + o1;
  const u64* b0 = Bp + o0;
  const u64* b1 = Bp + o1;
  const RowSt st(T3 + r * N);
  if (square) {
    if (c == 0)
      ntt_inv_gg(sm, [&](int x) { return mulmod(a0[x], a0[x], pr); }, st, V, pi);
    else if (c == 1)
      ntt_inv_gg(
          sm,
          [&](int x) {
            const u64 m = mulmod(a0[x], a1[x], pr);
            return addmod(m, m, pr.q);
          },
          st, V, pi);
    else
      ntt_inv_gg(sm, [&](int x) { return mulmod(a1[x], a1[x], pr); }, st, V, pi);
  } else {
    if (c == 0)
      ntt_inv_gg(sm, [&](int x) { return mulmod(a0[x], addmod(b0[x], cb, pr.q), pr); }, st, V, pi);
    else if (c == 1)
      ntt_inv_gg(
          sm,
          [&](int x) {
            u64 lo = 0, hi = 0;
            mac128(lo, hi, a0[x], b1[x]);
            mac128(lo, hi, a1[x], addmod(b0[x], cb, pr.q));
            return reduce128(hi, lo, pr);
          },
          st, V, pi);
    else
      ntt_inv_gg(sm, [&](int x) { return mulmod(a1[x], b1[x], pr); }, st, V, pi);
  }
}

// Relinearisation fused with the affine step after it: the block of row
// (l, c, p) of U[L][2][k][N] computes R_c = NTT(d_c) + sum_i NTT(d_i) *
// rlk_i[c] (the digit rows DG of k_relin_ntt, 128-bit sums, one reduction)
// and u = R_c + z * H on the load of the inverse NTT of U, stores u and the
// coefficient-form row.  The same words as k_relin_mac followed by
// k_axpy_intt, without R in memory.
template <int MT>
__global__ void __launch_bounds__(MT, relin_min_blocks(MT))
    k_relin_axpy_intt(DevView V, const u64* __restrict__ DG, const u64* __restrict__ rlk,
                      const u64* __restrict__ zres, const u64* __restrict__ H, u64* __restrict__ out, u64* coef) {
  extern __shared__ u64 sm[];
  const int N = V.N, k = V.k;
  const size_t r = blockIdx.x;
  const int p = (int)(r % k);
  const int c = (int)((r / k) % 2);
  const size_t l = r / ((size_t)2 * k);
  const DevPrime pr = V.pr[p];
  const u64 z = zres[p];
  const size_t gs = (size_t)k * N;  // digit row stride
  const u64* g = DG + l * (k + 2) * gs + (size_t)p * N;
  const u64* key = rlk + ((size_t)c * k + p) * N;  // rlk_i[c] at prime p: key + i * 2 * gs
  const u64* hr = H + r * N;
  u64* ur = out + r * N;
  ntt_inv_gg(
      sm,
      [&](int x) {
        u64 lo = g[(size_t)(k + c) * gs + x], hi = 0;
        for (int i = 0; i < k; ++i) mac128(lo, hi, g[(size_t)i * gs + x], __ldg(key + (size_t)i * 2 * gs + x));
        const u64 u = addmod(reduce128(hi, lo, pr), mulmod(z, hr[x], pr), pr.q);
        ur[x] = u;
        return u;
      },
      RowSt(coef + r * N), V, p);
}

// out = a + z * b (NTT form, rows [groups][k][N], z as k residues), fused
// with the inverse NTT of out into coef: the block of a row computes the
// row on the transform's load and also stores it (each element is loaded
// once).  coef may alias b: a block reads its row of b before it writes
// that row of coef.
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1)
    k_axpy_intt(DevView V, const u64* __restrict__ a, const u64* __restrict__ zres, const u64* b, u64* __restrict__ out,
                u64* coef) {
  extern __shared__ u64 sm[];
  const int N = V.N;
  const size_t r = blockIdx.x;
  const int p = (int)(r % V.k);
  const DevPrime pr = V.pr[p];
  const u64 z = zres[p];
  const u64* ar = a + r * N;
  const u64* br = b + r * N;
  u64* ur = out + r * N;
  u64* cr = coef + r * N;
  ntt_inv_gg(
      sm,
      [&](int x) {
        const u64 u = addmod(ar[x], mulmod(z, br[x], pr), pr.q);
        ur[x] = u;
        return u;
      },
      RowSt(cr), V, p);
}

// Lazy rescaling: X[c][pi][n] (+)= sum over layers l < L of component c of
// the tensor of (A_l, B_l), in NTT form over Q u B, each layer's tensor
// times its value plaintext VP[l][pi][n] when VP is given (labelled PSI /
// PSI-Sum).  The products of each (prime, point) are summed in 128 bits
// and reduced once per 16 layers (at most 32 products below 2^122 each
// stay below 2^127), so the sum is exact mod every prime; the integer it
// represents is the sum of the layers' exact integer tensors (times the
// values) as long as B holds it (sized at setup).
// Four blocks per SM (64 registers a thread, a few spilled): at the paper
// shape the sums of two 263-layer chunks took 0.27 ms against 0.31 ms with
// three blocks (80 registers), whose 1152 blocks left a half-empty last wave.
constexpr int TS_PTS = 64, TS_SLICES = 4;
__global__ void __launch_bounds__(TS_PTS * TS_SLICES, 4) k_tensor_sum(DevView V, const u64* __restrict__ AQ, const u64* __restrict__ AB,
                             const u64* __restrict__ BQ, const u64* __restrict__ BB, const u64* __restrict__ cstQ,
                             const u64* __restrict__ side, const u64* __restrict__ VP, u64* __restrict__ X, int L,
                             int square, int init) {
  // block: TS_PTS consecutive (prime, point) words x TS_SLICES slices of
  // the layers; each slice sums every TS_SLICES-th layer, and the slices'
  // residues are added at the end
  __shared__ u64 part[3][TS_SLICES][TS_PTS];
  const int N = V.N, k = V.k, kb = V.kb, np = k + kb;
  const int tp = threadIdx.x % TS_PTS, slice = threadIdx.x / TS_PTS;
  const size_t idx = (size_t)blockIdx.x * TS_PTS + tp;  // over np*N
  const bool active = idx < (size_t)np * N;  // every thread reaches the barrier below
  const int n = active ? (int)(idx % N) : 0;
  const int pi = active ? (int)(idx / N) : 0;
  const DevPrime pr = V.pr[pi];
  const bool inQ = pi < k;
  const int kk = inQ ? k : kb, pp = inQ ? pi : pi - k;
  const u64* A = inQ ? AQ : AB;
  const u64* Bp = inQ ? BQ : BB;
  const u64 cq = (inQ && cstQ) ? cstQ[pi] : 0;
  const size_t cs = (size_t)kk * N;  // component stride of the operands
  u64 s0l = 0, s0h = 0, s1l = 0, s1h = 0, s2l = 0, s2h = 0;
  int cnt = 0;
  for (int l = active ? slice : L; l < L; l += TS_SLICES) {
    const size_t o0 = ((size_t)l * 2 * kk + pp) * N + n;
    const u64 a0 = A[o0], a1 = A[o0 + cs];
    u64 b0 = a0, b1 = a1;
    if (!square) {
      b0 = Bp[o0];
      b1 = Bp[o0 + cs];
      if (inQ) {
        b0 = addmod(b0, cq, pr.q);
      } else if (side) {
        b0 = addmod(b0, side[(size_t)l * kb + pp], pr.q);
      }
    }
    if (VP) {
      const u64 v = VP[((size_t)l * np + pi) * N + n];
      u64 lo = 0, hi = 0;
      mac128(lo, hi, a0, b1);
      mac128(lo, hi, a1, b0);
      mac128(s0l, s0h, mulmod(a0, b0, pr), v);
      mac128(s1l, s1h, reduce128(hi, lo, pr), v);
      mac128(s2l, s2h, mulmod(a1, b1, pr), v);
    } else {
      mac128(s0l, s0h, a0, b0);
      mac128(s1l, s1h, a0, b1);
      mac128(s1l, s1h, a1, b0);
      mac128(s2l, s2h, a1, b1);
    }
    if ((++cnt & 15) == 0) {
      s0l = reduce128(s0h, s0l, pr);
      s1l = reduce128(s1h, s1l, pr);
      s2l = reduce128(s2h, s2l, pr);
      s0h = s1h = s2h = 0;
    }
  }
  part[0][slice][tp] = reduce128(s0h, s0l, pr);
  part[1][slice][tp] = reduce128(s1h, s1l, pr);
  part[2][slice][tp] = reduce128(s2h, s2l, pr);
  __syncthreads();
  if (slice == 0 && active) {
    u64* o = X + (size_t)pi * N + n;
    const size_t os = (size_t)np * N;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u64 d = part[c][0][tp];
#pragma unroll
      for (int sl = 1; sl < TS_SLICES; ++sl) d = addmod(d, part[c][sl][tp], pr.q);
      o[c * os] = init ? d : addmod(d, o[c * os], pr.q);
    }
  }
}

// ------------------------------------------------------ scale and round
// y = round(t x / Q) exactly: z = t x + (Q-1)/2, [z]_Q from the Q residues
// by Garner, y = (z - [z]_Q) / Q computed in B, y centred in B and mapped
// back to Q by Garner over B.
template <int K, int KB>
__global__ void k_scale_round(const __grid_constant__ RnsArgs A, const u64* __restrict__ T3, u64* __restrict__ D,
                              int L) {
  constexpr int MQ = K ? K : PEPSI_MAXQ, MB = KB ? KB : PEPSI_MAXB;
  const int N = A.N, k = K ? K : A.k, kb = KB ? KB : A.kb, np = k + kb;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over L*3*N
  if (idx >= (size_t)L * 3 * N) return;
  const int n = (int)(idx % N);
  const size_t lc = idx / N;
  const u64* in = T3 + lc * np * N + n;
  u64 z[MQ], v[MQ];
#pragma unroll
  for (int i = 0; i < MQ; ++i)
    if (K || i < k) {
      const u64 q = A.pr[i].q;
      z[i] = addmod(shoup(in[(size_t)i * N], A.rc.t_q[i], A.rc.t_qs[i], q), A.rc.qhalf_q[i], q);
    }
  garner_q<K>(A, z, v);
  u64 y[MB], u[MB];
#pragma unroll
  for (int j = 0; j < MB; ++j)
    if (KB || j < kb) {
      const DevPrime pb = A.pr[k + j];
      const u64 zb = addmod(shoup(in[(size_t)(k + j) * N], A.rc.t_b[j], A.rc.t_bs[j], pb.q), A.rc.qhalf_b[j], pb.q);
      const u64 zq = q_digits_mod_b<K>(A, v, false, j);
      y[j] = shoup(submod(zb, zq, pb.q), A.rc.qinv_b[j], A.rc.qinv_bs[j], pb.q);
    }
  garner_b<K, KB>(A, y, u);
  const bool neg = digits_greater<MB>(u, A.rc.bhalf_dig, kb);
  u64* out = D + lc * k * N + n;
#pragma unroll
  for (int i = 0; i < MQ; ++i)
    if (K || i < k) {
      const DevPrime pq = A.pr[i];
      // Horner over the B digits (each below 2^61): partial values below 2 q_i + 2^61
      u64 acc = u[kb - 1];
#pragma unroll
      for (int j = MB - 2; j >= 0; --j)
        if (KB || j < kb - 1) acc = shoup_lazy(acc, A.rc.bq[i][j], A.rc.bqs[i][j], pq.q) + u[j];
      const u64 r = barrett64(acc, pq);
      out[(size_t)i * N] = neg ? submod(r, A.rc.bmodq[i], pq.q) : r;
    }
}

// ---------------------------------------------------------- relinearise
// Phase 1, block per row of DG[L][k+2][k][N]: row (l, i, j) holds
// NTT_{q_j}([d2]_{q_i}) for digits i < k, and NTT_{q_j}(d0), NTT_{q_j}(d1)
// for i = k, k+1.
template <int MT>
__global__ void __launch_bounds__(MT, relin_min_blocks(MT)) k_relin_ntt(DevView V, const u64* __restrict__ D, u64* __restrict__ DG) {
  extern __shared__ u64 sm[];
  const int N = V.N, k = V.k;
  const size_t r = blockIdx.x;
  const int j = (int)(r % k);
  const int i = (int)((r / k) % (k + 2));
  const size_t l = r / ((size_t)k * (k + 2));
  const DevPrime pj = V.pr[j];
  const u64* row = i < k ? D + ((l * 3 + 2) * k + i) * N : D + ((l * 3 + (i - k)) * k + j) * N;
  u64* out = DG + r * N;
  ntt_fwd_gg(
      sm,
      [&](int x) {
        const u64 w = row[x];
        return w >= pj.q ? barrett64(w, pj) : w;
      },
      RowSt(out), V, j);
}
// Phase 2, thread per (l, j, n): R_c = NTT(d_c) + sum_i NTT(d_i) * rlk_i[c],
// 128-bit lazy sums, one Barrett reduction per output.
__global__ void k_relin_mac(DevView V, const u64* __restrict__ DG, const u64* __restrict__ rlk, u64* __restrict__ R,
                            int L) {
  const int N = V.N, k = V.k;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over L*k*N
  if (idx >= (size_t)L * k * N) return;
  const int n = (int)(idx % N);
  const int j = (int)((idx / N) % k);
  const size_t l = idx / ((size_t)k * N);
  const DevPrime pj = V.pr[j];
  const u64* g = DG + l * (k + 2) * k * N + (size_t)j * N + n;
  const size_t gs = (size_t)k * N;
  u64 lo0 = g[(size_t)k * gs], hi0 = 0, lo1 = g[(size_t)(k + 1) * gs], hi1 = 0;
  for (int i = 0; i < k; ++i) {
    const u64 d = g[(size_t)i * gs];
    mac128(lo0, hi0, d, __ldg(rlk + (((size_t)i * 2 + 0) * k + j) * N + n));
    mac128(lo1, hi1, d, __ldg(rlk + (((size_t)i * 2 + 1) * k + j) * N + n));
  }
  u64* o = R + ((l * 2) * k + j) * N + n;
  o[0] = reduce128(hi0, lo0, pj);
  o[(size_t)k * N] = reduce128(hi1, lo1, pj);
}

// ------------------------------------------------------------ pointwise
__global__ void k_axpy(DevView V, const u64* __restrict__ a, const u64* __restrict__ zres, const u64* __restrict__ b,
                       u64* out, size_t total) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int p = (int)((idx / V.N) % V.k);
  const DevPrime pr = V.pr[p];
  out[idx] = addmod(a[idx], mulmod(zres[p], b[idx], pr), pr.q);
}

__global__ void k_accum(DevView V, const u64* __restrict__ D, int L, u64* acc, int init) {
  const size_t per = (size_t)3 * V.k * V.N;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per) return;
  const u64 q = V.pr[(idx / V.N) % V.k].q;
  u64 s = init ? 0 : acc[idx];
  for (int l = 0; l < L; ++l) s = addmod(s, D[(size_t)l * per + idx], q);
  acc[idx] = s;
}

// ---------------------------------------------------------------- client
// round(Q m / t) mod q_p for m in [0, t): floor(Q/t) m + round((Q mod t) m / t)
__device__ __forceinline__ u64 delta_of(const DevView& V, u64 m, int p, u64 t) {
  const DevPrime pq = V.pr[p];
  const u64 a = shoup(m, V.rc->qdt_q[p], V.rc->qdt_qs[p], pq.q);
  const u64 b = (V.rc->qmt * m + (t - 1) / 2) / t;
  return addmod(a, b % pq.q, pq.q);
}
__device__ __forceinline__ u64 smod_dev(i64 v, u64 q) { return v >= 0 ? (u64)v : q - (u64)(-v); }

// Block per ciphertext j: encode bit plane j, then for each prime sample
// a, compute c0 = e - a s + round(Q m / t), c1 = a (coefficient form).
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_encrypt(DevView V, const uint16_t* __restrict__ pos, int h, const u64* __restrict__ s_ntt, u64 seed,
                          u64 idx0, u64* cts) {
  extern __shared__ u64 sm[];
  const int N = V.N, k = V.k, j = blockIdx.x;
  u64* poly = sm;
  u32* mbuf = reinterpret_cast<u32*>(sm + N);
  const u64 t = V.pr[V.tidx].q;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int s = (int)brev_bits(i, V.logN);
    const uint16_t* ps = pos + (size_t)s * h;
    u64 bit = 0;
    if (ps[0] != PEPSI_CW_NONE)
      for (int r = 0; r < h; ++r) bit |= (ps[r] == j);
    poly[nsw(i)] = bit;
  }
  __syncthreads();
  ntt_inv_view(poly, V, V.tidx);
  for (int i = threadIdx.x; i < N; i += blockDim.x) mbuf[i] = (u32)poly[nsw(i)];
  __syncthreads();
  const u64 key_e = stream_key(seed, make_stream(STREAM_ENC_E, idx0 + j, 0));
  for (int p = 0; p < k; ++p) {
    const DevPrime pq = V.pr[p];
    const u64 key_a = stream_key(seed, make_stream(STREAM_ENC_A, idx0 + j, p));
    u64* c0 = cts + (((size_t)j * 2 + 0) * k + p) * N;
    u64* c1 = cts + (((size_t)j * 2 + 1) * k + p) * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const u64 a = sample_uniform(key_a, i, pq.q);
      c1[i] = a;
      poly[nsw(i)] = a;
    }
    __syncthreads();
    ntt_fwd_view(poly, V, p);
    const u64* sr = s_ntt + (size_t)p * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) poly[nsw(i)] = mulmod(poly[nsw(i)], sr[i], pq);
    __syncthreads();
    ntt_inv_view(poly, V, p);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const u64 e = smod_dev(sample_cbd21(key_e, i), pq.q);
      c0[i] = addmod(submod(e, poly[nsw(i)], pq.q), delta_of(V, mbuf[i], p, t), pq.q);
    }
    __syncthreads();
  }
}

__global__ void k_keygen_s(DevView V, u64 seed, int8_t* s) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= V.N) return;
  const u64 key = stream_key(seed, make_stream(STREAM_SK, 0, 0));
  s[n] = (int8_t)((int)sample_uniform(key, n, 3) - 1);
}
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_keygen_sntt(DevView V, const int8_t* __restrict__ s, u64* s_ntt) {
  extern __shared__ u64 sm[];
  const int p = blockIdx.x, N = V.N;
  const u64 q = V.pr[p].q;
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[nsw(i)] = smod_dev(s[i], q);
  __syncthreads();
  ntt_fwd_view(sm, V, p);
  for (int i = threadIdx.x; i < N; i += blockDim.x) s_ntt[(size_t)p * N + i] = sm[nsw(i)];
}
// Block (digit i, prime j): rlk_i = (-a_i s + e_i + g_i s^2, a_i) in NTT form,
// g_i = 1 mod q_i and 0 mod q_j for j != i.
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_keygen_rlk(DevView V, u64 seed, const u64* __restrict__ s_ntt, u64* rlk) {
  extern __shared__ u64 sm[];
  const int N = V.N, k = V.k;
  const int i = blockIdx.x / k, j = blockIdx.x % k;
  const DevPrime pj = V.pr[j];
  u64* r0 = rlk + (((size_t)i * 2 + 0) * k + j) * N;
  u64* r1 = rlk + (((size_t)i * 2 + 1) * k + j) * N;
  const u64 key_e = stream_key(seed, make_stream(STREAM_RLK_E, i, 0));
  const u64 key_a = stream_key(seed, make_stream(STREAM_RLK_A, i, j));
  for (int x = threadIdx.x; x < N; x += blockDim.x) sm[nsw(x)] = smod_dev(sample_cbd21(key_e, x), pj.q);
  __syncthreads();
  ntt_fwd_view(sm, V, j);
  for (int x = threadIdx.x; x < N; x += blockDim.x) r0[x] = sm[nsw(x)];
  __syncthreads();
  for (int x = threadIdx.x; x < N; x += blockDim.x) sm[nsw(x)] = sample_uniform(key_a, x, pj.q);
  __syncthreads();
  ntt_fwd_view(sm, V, j);
  const u64* sr = s_ntt + (size_t)j * N;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const u64 a = sm[nsw(x)], sv = sr[x];
    u64 v = submod(r0[x], mulmod(a, sv, pj), pj.q);
    if (i == j) v = addmod(v, mulmod(sv, sv, pj), pj.q);
    r0[x] = v;
    r1[x] = a;
  }
}

// Decryption, step 1: z = c0 + c1 s per prime (coefficient form).
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_dec_z(DevView V, const u64* __restrict__ ct, const u64* __restrict__ s_ntt, u64* z) {
  extern __shared__ u64 sm[];
  const int p = blockIdx.x, N = V.N, k = V.k;
  const DevPrime pq = V.pr[p];
  const u64* c1 = ct + ((size_t)k + p) * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[nsw(i)] = c1[i];
  __syncthreads();
  ntt_fwd_view(sm, V, p);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[nsw(i)] = mulmod(sm[nsw(i)], s_ntt[(size_t)p * N + i], pq);
  __syncthreads();
  ntt_inv_view(sm, V, p);
  for (int i = threadIdx.x; i < N; i += blockDim.x) z[(size_t)p * N + i] = addmod(sm[nsw(i)], ct[(size_t)p * N + i], pq.q);
}
// Step 2, per coefficient: m = round(t z / Q) mod t exactly (Garner of
// w = t z + (Q-1)/2 over Q, then (w - [w]_Q)/Q mod t), and the noise
// |[t z]_Q| (centred) as a double, maximised over coefficients.
__global__ void k_dec_coef(const __grid_constant__ RnsArgs A, DevView V, const u64* __restrict__ z, u32* m,
                           unsigned long long* maxr) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = V.N, k = V.k;
  const RnsConst* rc = &A.rc;
  const u64 t = V.pr[V.tidx].q;
  double rabs = 0.0;
  if (n < N) {
    u64 w[PEPSI_MAXQ], v[PEPSI_MAXQ];
#pragma unroll
    for (int i = 0; i < PEPSI_MAXQ; ++i)
      if (i < k) {
        const u64 q = V.pr[i].q;
        w[i] = addmod(shoup(z[(size_t)i * N + n], rc->t_q[i], rc->t_qs[i], q), rc->qhalf_q[i], q);
      }
    garner_q<0>(A, w, v);
    u64 wq = 0;
#pragma unroll
    for (int l = 0; l < PEPSI_MAXQ; ++l)
      if (l < k) wq = (wq + (v[l] % t) * rc->pq_t[l]) % t;
    m[n] = (u32)(((rc->qhalf_t + t - wq) % t) * rc->qinv_t % t);
#pragma unroll
    for (int i = 0; i < PEPSI_MAXQ; ++i)
      if (i < k) w[i] = shoup(z[(size_t)i * N + n], rc->t_q[i], rc->t_qs[i], V.pr[i].q);
    garner_q<0>(A, w, v);
    if (digits_greater<PEPSI_MAXQ>(v, rc->qhalf_dig, k)) {
#pragma unroll
      for (int i = 0; i < PEPSI_MAXQ; ++i)
        if (i < k) w[i] = w[i] ? V.pr[i].q - w[i] : 0;
      garner_q<0>(A, w, v);
    }
#pragma unroll
    for (int l = 0; l < PEPSI_MAXQ; ++l)
      if (l < k) rabs += (double)v[l] * rc->pq_d[l];
  }
  // block max, then one atomic per block (positive doubles order like u64)
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) rabs = fmax(rabs, __shfl_down_sync(0xffffffffu, rabs, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rabs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) b = fmax(b, red[i]);
    atomicMax(maxr, (unsigned long long)__double_as_longlong(b));
  }
}
// Step 3: slots = values of m at psi_t^(2s+1): forward NTT mod t, slot s in position brev(s).
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_dec_slots(DevView V, const u32* __restrict__ m, u32* slots) {
  extern __shared__ u64 sm[];
  const int N = V.N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm[nsw(i)] = m[i];
  __syncthreads();
  ntt_fwd_view(sm, V, V.tidx);
  for (int s = threadIdx.x; s < N; s += blockDim.x) slots[s] = (u32)sm[nsw(brev_bits(s, V.logN))];
}

// Modulus switching of the response to the first r primes: per
// coefficient, with z = c + (Q'-1)/2, [z]_{Q'} from Garner over the dropped
// primes, y = (z - [z]_{Q'}) / Q' mod q_i = round(c~ / Q') for any
// representative c of the residue class mod Q (Q' odd, no ties).
__global__ void k_modswitch(const __grid_constant__ ModSwitchArgs M, DevView V, const u64* __restrict__ in,
                            u64* __restrict__ out, size_t n) {
  const int N = V.N, k = M.k, r = M.r, m = k - r;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over n*2*N
  if (idx >= n * 2 * N) return;
  const int x = (int)(idx % N);
  const size_t cc = idx / N;  // ciphertext * 2 + component
  const u64* src = in + cc * k * N + x;
  u64 v[PEPSI_MAXQ];
#pragma unroll
  for (int j = 0; j < PEPSI_MAXQ; ++j) {
    if (j < m) {
      const DevPrime d = V.pr[r + j];
      u64 z = addmod(src[(size_t)(r + j) * N], M.h[r + j], d.q);
#pragma unroll
      for (int l = 0; l < PEPSI_MAXQ; ++l)
        if (l < j) z = mulmod(submod(z, barrett64(v[l], d), d.q), M.ginv[j][l], d);
      v[j] = z;
    }
  }
  u64* dst = out + cc * r * N + x;
  for (int i = 0; i < r; ++i) {
    const DevPrime qi = V.pr[i];
    u64 S = 0;
#pragma unroll
    for (int j = 0; j < PEPSI_MAXQ; ++j)
      if (j < m) S = addmod(S, mulmod(barrett64(v[j], qi), M.pw[i][j], qi), qi.q);
    dst[(size_t)i * N] = mulmod(submod(addmod(src[(size_t)i * N], M.h[i], qi.q), S, qi.q), M.qdinv[i], qi);
  }
}

// Cardinality mask (Algorithm 5): r_s uniform in Z_t for s < N-1,
// r_{N-1} = -sum; c0 += round(Q Encode(r) / t).  One block.
__global__ void __launch_bounds__(NTT_MAX_THREADS, 1) k_mask(DevView V, u64 seed, u64* ct) {
  extern __shared__ u64 sm[];
  __shared__ u64 red[32];
  const int N = V.N, k = V.k;
  const u64 t = V.pr[V.tidx].q;
  const u64 key = stream_key(seed, make_stream(STREAM_MASK, 0, 0));
  u64 part = 0;
  for (int s = threadIdx.x; s < N - 1; s += blockDim.x) {
    const u64 r = sample_uniform(key, s, t);
    sm[nsw(brev_bits(s, V.logN))] = r;
    part += r;
  }
  part %= t;
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part % t;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 sum = 0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) sum = (sum + red[i]) % t;
    sm[nsw(brev_bits(N - 1, V.logN))] = (t - sum) % t;
  }
  __syncthreads();
  ntt_inv_view(sm, V, V.tidx);
  for (int p = 0; p < k; ++p) {
    const u64 q = V.pr[p].q;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      u64* c = ct + (size_t)p * N + n;
      *c = addmod(*c, delta_of(V, sm[nsw(n)], p, t), q);
    }
  }
}

inline unsigned grid_for(size_t total, int threads) { return (unsigned)((total + threads - 1) / threads); }

}  // namespace

// ------------------------------------------------------------ launchers
void launch_ntt(const DevView& V, bool fwd, const u64* src, u64* dst, size_t outer, int np, int p0, size_t src_os,
                size_t dst_os, cudaStream_t st, bool split_out, u32* sums) {
  const size_t rows = outer * (size_t)np;
  if (!rows) return;
  const size_t smem = (size_t)V.N * sizeof(u64);
  if (fwd && split_out)
    k_ntt<true, true><<<(unsigned)rows, xform_threads(V, rows), smem, st>>>(V, src, dst, np, p0, src_os, dst_os, sums);
  else if (fwd)
    k_ntt<true><<<(unsigned)rows, xform_threads(V, rows), smem, st>>>(V, src, dst, np, p0, src_os, dst_os, nullptr);
  else
    k_ntt<false><<<(unsigned)rows, xform_threads(V, rows), smem, st>>>(V, src, dst, np, p0, src_os, dst_os, nullptr);
}

void launch_cuckoo_round(const u32* bins3, u32 m, u32 nbins, u32 gamma, u32* claim, int32_t* slot_item, u32* load,
                         u32* evictions, uint8_t* state, uint8_t* choice, u32* unplaced, cudaStream_t st) {
  if (!m) return;
  k_ck_claim<<<grid_for(m, 256), 256, 0, st>>>(bins3, state, choice, m, claim);
  k_ck_resolve<<<grid_for(nbins, 256), 256, 0, st>>>(nbins, gamma, claim, slot_item, load, evictions, state, choice);
  k_ck_advance<<<grid_for(m, 256), 256, 0, st>>>(m, state, choice, unplaced);
}

void launch_cw_unrank(const u64* T, size_t count, const u64* binom, int ell, int h, uint16_t* pos, cudaStream_t st) {
  if (!count) return;
  k_cw_unrank<<<grid_for(count, 256), 256, 0, st>>>(T, count, binom, ell, h, pos);
}

static int ptgen_jc(int N) { return N >= 16384 ? 8 : 32; }
static size_t ptgen_smem(int N) {
  const int words = N / 32 > 0 ? N / 32 : 1;
  return (size_t)N * 8 + (size_t)N * 4 + (size_t)ptgen_jc(N) * words * 4;
}

void launch_ptgen(const DevView& V, const uint16_t* pos, int L, int ell, int h, u64* P, cudaStream_t st) {
  if (L <= 0) return;
  const int JC = ptgen_jc(V.N);
  dim3 grid((ell + JC - 1) / JC, L);
  k_ptgen<<<grid, ntt_threads(V.N), ptgen_smem(V.N), st>>>(V, pos, ell, h, JC, P);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}
// 3-D tensor of elements of esz bytes: dims (d0, d1, d2), row strides s1, s2 in elements, box (b0, b1, b2)
bool encode3d_t(CUtensorMap* tm, CUtensorMapDataType dt, int esz, const void* base, u64 d0, u64 d1, u64 d2, u64 s1,
                u64 s2, u32 b0, u32 b1, u32 b2) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {s1 * esz, s2 * esz};
  const cuuint32_t box[3] = {b0, b1, b2};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(tm, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
bool encode3d(CUtensorMap* tm, const u64* base, u64 d0, u64 d1, u64 d2, u64 s1, u64 s2, u32 b0, u32 b1, u32 b2) {
  return encode3d_t(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 8, base, d0, d1, d2, s1, s2, b0, b1, b2);
}
// Tensor maps of the plaintext tiles of L layers [L][ell][kN]: tm[0] the words, or
// tm[0..2] the three planes of the 7-byte format (tm[1], tm[2] copies of tm[0] otherwise).
bool encode_plain(CUtensorMap tm[3], const PlainTab& P, u64 kN, int ell, int L, u32 tn, u32 js, u32 lb) {
  const u64 s2 = (u64)ell * kN;
  if (!P.packed()) {
    if (!encode3d(&tm[0], P.w, kN, ell, L, kN, s2, tn, js, lb)) return false;
    tm[1] = tm[2] = tm[0];
    return true;
  }
  return encode3d_t(&tm[0], CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, P.a, kN, ell, L, kN, s2, tn, js, lb) &&
         encode3d_t(&tm[1], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, P.b, kN, ell, L, kN, s2, tn, js, lb) &&
         encode3d_t(&tm[2], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, P.c, kN, ell, L, kN, s2, tn, js, lb);
}
bool encode4d(CUtensorMap* tm, const u64* base, u64 d0, u64 d1, u64 d2, u64 d3, u64 s1, u64 s2, u64 s3, u32 b0,
              u32 b1, u32 b2, u32 b3) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {d0, d1, d2, d3};
  const cuuint64_t strides[3] = {s1 * 8, s2 * 8, s3 * 8};
  const cuuint32_t box[4] = {b0, b1, b2, b3};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<u64*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

namespace {
template <int QB, int RG, int WPS, bool P7>
void mac_multi_go(const DevView& V, const CUtensorMap (&tmP)[3], const MacRequests& rq, int ell, int L,
                  int fold_stages, int* err, cudaStream_t st) {
  using TL = macq::Tile<WPS>;
  const u64 kN = (u64)V.k * V.N;
  dim3 grid((L + TL::LB - 1) / TL::LB, (unsigned)((kN + TL::TN - 1) / TL::TN));
  k_mac_multi<QB, RG, WPS, P7><<<grid, macq::threads(RG), macq::smem<QB, WPS, P7>(), st>>>(
      V, tmP[0], tmP[1], tmP[2], rq, ell, L, fold_stages, err);
}
// groups: 1 = every consumer thread serves all requests; 2 = two groups of
// warps serve half of them each (2 or 4 requests)
template <int WPS, bool P7>
void mac_multi_q(int nq, int groups, const DevView& V, const CUtensorMap (&tmP)[3], const MacRequests& rq, int ell,
                 int L, int fold_stages, int* err, cudaStream_t st) {
  switch (nq * 4 + (groups == 2 && nq != 3 ? 2 : 1)) {
    case 2 * 4 + 1: mac_multi_go<2, 1, WPS, P7>(V, tmP, rq, ell, L, fold_stages, err, st); break;
    case 2 * 4 + 2: mac_multi_go<2, 2, WPS, P7>(V, tmP, rq, ell, L, fold_stages, err, st); break;
    case 3 * 4 + 1: mac_multi_go<3, 1, WPS, P7>(V, tmP, rq, ell, L, fold_stages, err, st); break;
    case 4 * 4 + 1: mac_multi_go<4, 1, WPS, P7>(V, tmP, rq, ell, L, fold_stages, err, st); break;
    default: mac_multi_go<4, 2, WPS, P7>(V, tmP, rq, ell, L, fold_stages, err, st); break;
  }
}
}  // namespace

cudaError_t launch_mac_requests(const DevView& V, int nq, const u64* const* C, const PlainTab& P, u64* const* H,
                                int ell, int L, int fold, int* err, cudaStream_t st, int tile_points, int groups) {
  if (L <= 0 || nq <= 0) return cudaSuccess;
  if (nq > macq::QMAX || (tile_points != 32 && tile_points != 64)) return cudaErrorInvalidValue;
  if (nq == 1) return launch_mac(V, C[0], P, H[0], ell, L, fold, err, st);  // one request: the single-request kernel
  const u64 kN = (u64)V.k * V.N;
  const int wps = tile_points / 32;
  const u32 tn = (u32)tile_points, lb = (u32)(macq::GROUP_WARPS / wps * macq::LPT);
  CUtensorMap tmP[3];
  MacRequests rq;
  memset(&rq, 0, sizeof(rq));
  if (!encode_plain(tmP, P, kN, ell, L, tn, macq::JS, lb)) return cudaErrorInvalidValue;
  for (int q = 0; q < nq; ++q) {
    if (!encode3d(&rq.c[q], C[q], kN, 2, ell, kN, 2 * kN, tn, 2, macq::JS) ||
        !encode3d_t(&rq.s[q], CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, request_sums(C[q], ell, kN), kN, 2, ell, kN, 2 * kN, tn,
                    2, macq::JS))
      return cudaErrorInvalidValue;
    rq.h[q] = H[q];
  }
  const int fold_stages = fold / macq::JS > 0 ? fold / macq::JS : 1;
  if (wps == 1) {
    if (P.packed())
      mac_multi_q<1, true>(nq, groups, V, tmP, rq, ell, L, fold_stages, err, st);
    else
      mac_multi_q<1, false>(nq, groups, V, tmP, rq, ell, L, fold_stages, err, st);
  } else {
    if (P.packed())
      mac_multi_q<2, true>(nq, groups, V, tmP, rq, ell, L, fold_stages, err, st);
    else
      mac_multi_q<2, false>(nq, groups, V, tmP, rq, ell, L, fold_stages, err, st);
  }
  return cudaSuccess;
}

cudaError_t launch_mac_multi(const DevView& V, const u64* C, int nq, const PlainTab& P, u64* H, size_t hq, int ell,
                             int L, int fold, int* err, cudaStream_t st, int tile_points, int groups) {
  if (nq <= 0 || nq > macq::QMAX) return nq <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  const u64* cq[macq::QMAX];
  u64* hqv[macq::QMAX];
  for (int q = 0; q < nq; ++q) {
    cq[q] = C + (size_t)q * request_prepared_words(ell, (size_t)V.k * V.N);
    hqv[q] = H + (size_t)q * hq;
  }
  return launch_mac_requests(V, nq, cq, P, hqv, ell, L, fold, err, st, tile_points, groups);
}

cudaError_t launch_mac(const DevView& V, const u64* C, const PlainTab& P, u64* H, int ell, int L, int fold, int* err,
                       cudaStream_t st, int j0, int nj, bool acc_in) {
  if (L <= 0) return cudaSuccess;
  if (nj < 0) nj = ell - j0;
  if (j0 < 0 || nj <= 0 || j0 + nj > ell || (j0 % mac::JS) || (j0 + nj < ell && nj % mac::JS))
    return cudaErrorInvalidValue;
  const u64 kN = (u64)V.k * V.N;
  CUtensorMap tmP[3], tmC, tmS;
  if (!encode_plain(tmP, P, kN, ell, L, mac::TN, mac::JS, mac::LB) ||
      !encode3d(&tmC, C, kN, 2, ell, kN, 2 * kN, mac::TN, 2, mac::JS) ||
      !encode3d_t(&tmS, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, request_sums(C, ell, kN), kN, 2, ell, kN, 2 * kN, mac::TN, 2,
                  mac::JS))
    return cudaErrorInvalidValue;
  const int fold_stages = fold / mac::JS > 0 ? fold / mac::JS : 1;
  dim3 grid((L + mac::LB - 1) / mac::LB, (unsigned)((kN + mac::TN - 1) / mac::TN));
  if (P.packed())
    k_mac<true><<<grid, mac::THREADS, mac::smem<true>(), st>>>(V, tmP[0], tmP[1], tmP[2], tmC, tmS, H, j0, nj, L,
                                                               fold_stages, acc_in ? 1 : 0, err);
  else
    k_mac<false><<<grid, mac::THREADS, mac::smem<false>(), st>>>(V, tmP[0], tmP[1], tmP[2], tmC, tmS, H, j0, nj, L,
                                                                 fold_stages, acc_in ? 1 : 0, err);
  return cudaSuccess;
}

void launch_pack7(const DevView& V, const u64* src, size_t count, u32* a, uint16_t* b, uint8_t* c, cudaStream_t st) {
  if (!count) return;
  k_pack7<<<grid_for(count, 256), 256, 0, st>>>(V, src, count, a, b, c);
}
void launch_unpack7(const u32* a, const uint16_t* b, const uint8_t* c, size_t count, u64* out, cudaStream_t st) {
  if (!count) return;
  k_unpack7<<<grid_for(count, 256), 256, 0, st>>>(a, b, c, count, out);
}

void launch_split(const DevView& V, u64* x, size_t groups, bool to, cudaStream_t st) {
  const size_t total = groups * V.k * V.N;
  if (!total) return;
  k_split<<<grid_for(total, 256), 256, 0, st>>>(V, x, total, to ? 1 : 0);
}

// instantiate F<K, KB> for the prime counts in use, else the run-time generic version
#define PEPSI_RNS_DISPATCH(V, LAUNCH)                 \
  switch ((V).k * 16 + (V).kb) {                      \
    case 3 * 16 + 3: LAUNCH(3, 3); break;             \
    case 4 * 16 + 4: LAUNCH(4, 4); break;             \
    case 4 * 16 + 5: LAUNCH(4, 5); break;             \
    case 8 * 16 + 8: LAUNCH(8, 8); break;             \
    case 8 * 16 + 9: LAUNCH(8, 9); break;             \
    default: LAUNCH(0, 0); break;                     \
  }

void launch_lift(const DevView& V, const u64* src, u64* dstB, int L, const u64* cst, u64* side, cudaStream_t st) {
  const size_t total = (size_t)L * 2 * V.N;
  if (!total) return;
#define LIFT(KQ, KBB) k_lift<KQ, KBB><<<grid_for(total, 128), 128, 0, st>>>(*V.host_args, src, dstB, L, cst, side)
  PEPSI_RNS_DISPATCH(V, LIFT)
#undef LIFT
}

void launch_tensor_intt(const DevView& V, const u64* AQ, const u64* AB, const u64* BQ, const u64* BB,
                        const u64* cstQ, const u64* side, u64* T3, int L, bool square, cudaStream_t st) {
  const size_t rows = (size_t)L * 3 * (V.k + V.kb);
  if (!rows) return;
  k_tensor_intt<<<(unsigned)rows, xform_threads(V, rows), (size_t)V.N * 8, st>>>(V, AQ, AB, BQ, BB, cstQ, side, T3,
                                                                          square ? 1 : 0);
}

void launch_tensor_sum(const DevView& V, const u64* AQ, const u64* AB, const u64* BQ, const u64* BB,
                       const u64* cstQ, const u64* side, const u64* VP, u64* X, int L, bool square, bool init,
                       cudaStream_t st) {
  const size_t total = (size_t)(V.k + V.kb) * V.N;
  k_tensor_sum<<<(unsigned)((total + TS_PTS - 1) / TS_PTS), TS_PTS * TS_SLICES, 0, st>>>(V, AQ, AB, BQ, BB, cstQ, side, VP, X, L,
                                                                          square ? 1 : 0, init ? 1 : 0);
}

void launch_valgen(const DevView& V, const u32* vals, int L, u64* VP, cudaStream_t st) {
  if (L <= 0) return;
  k_valgen<<<L, ntt_threads(V.N), (size_t)V.N * 12, st>>>(V, vals, VP);
}

// Value-weighted layer sum with per-layer rounding: acc[c][p][n] (+)=
// sum_{l<L} D_l[c][p][n] * VP_l[p][n] mod q_p, D in NTT form over Q.  One
// product below 2^122 per layer; the 128-bit sums are reduced every 32.
__global__ void k_accum_val(DevView V, const u64* __restrict__ D, const u64* __restrict__ VP, int L, u64* acc,
                            int init) {
  const int N = V.N, k = V.k, np = V.k + V.kb;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // over 3*k*N
  if (idx >= (size_t)3 * k * N) return;
  const int n = (int)(idx % N);
  const int p = (int)((idx / N) % k);
  const int c = (int)(idx / ((size_t)k * N));
  const DevPrime pr = V.pr[p];
  u64 lo = 0, hi = 0;
  for (int l = 0; l < L; ++l) {
    mac128(lo, hi, D[(((size_t)l * 3 + c) * k + p) * N + n], VP[((size_t)l * np + p) * N + n]);
    if ((l & 31) == 31) {
      lo = reduce128(hi, lo, pr);
      hi = 0;
    }
  }
  const u64 r = reduce128(hi, lo, pr);
  acc[idx] = init ? r : addmod(r, acc[idx], pr.q);
}

void launch_accum_val(const DevView& V, const u64* D, const u64* VP, int L, u64* acc, bool init, cudaStream_t st) {
  const size_t total = (size_t)3 * V.k * V.N;
  k_accum_val<<<grid_for(total, 256), 256, 0, st>>>(V, D, VP, L, acc, init ? 1 : 0);
}

void launch_scale_round(const DevView& V, const u64* T3, u64* D, int L, cudaStream_t st) {
  const size_t total = (size_t)L * 3 * V.N;
  if (!total) return;
#define SCALE(KQ, KBB) k_scale_round<KQ, KBB><<<grid_for(total, 128), 128, 0, st>>>(*V.host_args, T3, D, L)
  PEPSI_RNS_DISPATCH(V, SCALE)
#undef SCALE
}

void launch_relin_digits(const DevView& V, const u64* D, u64* DG, int L, cudaStream_t st) {
  if (L <= 0) return;
  const size_t rows = (size_t)L * (V.k + 2) * V.k;
  const int nt = xform_threads(V, rows);
  if (nt <= 256)
    k_relin_ntt<256><<<(unsigned)rows, nt, (size_t)V.N * 8, st>>>(V, D, DG);
  else
    k_relin_ntt<NTT_MAX_THREADS><<<(unsigned)rows, nt, (size_t)V.N * 8, st>>>(V, D, DG);
}

void launch_relin(const DevView& V, const u64* D, const u64* rlk, u64* DG, u64* R, int L, cudaStream_t st) {
  if (L <= 0) return;
  launch_relin_digits(V, D, DG, L, st);
  k_relin_mac<<<grid_for((size_t)L * V.k * V.N, 256), 256, 0, st>>>(V, DG, rlk, R, L);
}

void launch_relin_axpy_intt(const DevView& V, const u64* DG, const u64* rlk, const u64* zres, const u64* H, u64* out,
                            u64* coef, int L, cudaStream_t st) {
  const size_t rows = (size_t)L * 2 * V.k;
  if (!rows) return;
  const int nt = xform_threads(V, rows);
  if (nt <= 256)
    k_relin_axpy_intt<256><<<(unsigned)rows, nt, (size_t)V.N * 8, st>>>(V, DG, rlk, zres, H, out, coef);
  else
    k_relin_axpy_intt<NTT_MAX_THREADS><<<(unsigned)rows, nt, (size_t)V.N * 8, st>>>(V, DG, rlk, zres, H, out, coef);
}

void launch_axpy_intt(const DevView& V, const u64* a, const u64* zres, const u64* b, u64* out, u64* coef,
                      size_t groups, cudaStream_t st) {
  const size_t rows = groups * V.k;
  if (!rows) return;
  k_axpy_intt<<<(unsigned)rows, xform_threads(V, rows), (size_t)V.N * 8, st>>>(V, a, zres, b, out, coef);
}

void launch_axpy(const DevView& V, const u64* a, const u64* zres, const u64* b, u64* out, size_t groups,
                 cudaStream_t st) {
  const size_t total = groups * V.k * V.N;
  if (!total) return;
  k_axpy<<<grid_for(total, 256), 256, 0, st>>>(V, a, zres, b, out, total);
}

void launch_accum(const DevView& V, const u64* D, int L, u64* acc, bool init, cudaStream_t st) {
  const size_t total = (size_t)3 * V.k * V.N;
  k_accum<<<grid_for(total, 256), 256, 0, st>>>(V, D, L, acc, init ? 1 : 0);
}

void launch_encrypt(const DevView& V, const uint16_t* pos, int ell, int h, const u64* s_ntt, u64 seed, u64 idx0,
                    u64* cts, cudaStream_t st) {
  if (ell <= 0) return;
  k_encrypt<<<ell, ntt_threads(V.N), (size_t)V.N * 12, st>>>(V, pos, h, s_ntt, seed, idx0, cts);
}

void launch_keygen(const DevView& V, u64 seed, int8_t* s, u64* s_ntt, u64* rlk, cudaStream_t st) {
  k_keygen_s<<<grid_for(V.N, 256), 256, 0, st>>>(V, seed, s);
  k_keygen_sntt<<<V.k, ntt_threads(V.N), (size_t)V.N * 8, st>>>(V, s, s_ntt);
  k_keygen_rlk<<<V.k * V.k, ntt_threads(V.N), (size_t)V.N * 8, st>>>(V, seed, s_ntt, rlk);
}

void launch_modswitch(const DevView& V, const ModSwitchArgs& M, const u64* in, u64* out, size_t n, cudaStream_t st) {
  const size_t total = n * 2 * V.N;
  if (!total) return;
  k_modswitch<<<grid_for(total, 256), 256, 0, st>>>(M, V, in, out, n);
}

// Test of the multiply-accumulate's bounded wait (mbar_wait_bounded): one thread waits on an mbarrier that
// needs one arrival.  With arrive != 0 it arrives first and the wait
// completes; with arrive == 0 nothing completes the phase, the wait gives
// up after about one second and the kernel sets *err and returns, as the
// multiply-accumulate does when its copies never land.
__global__ void k_wait_probe(int arrive, int* err) {
  __shared__ __align__(8) u64 bar;
  const u32 addr = (u32)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    mbar_init(addr, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) mbar_arrive(addr);
    if (!mbar_wait_bounded(addr, 0)) atomicExch(err, 1);
  }
}

void launch_wait_probe(int arrive, int* err, cudaStream_t st) { k_wait_probe<<<1, 32, 0, st>>>(arrive, err); }

void launch_decrypt(const DevView& V, const u64* ct, const u64* s_ntt, u64* zbuf, u32* mbuf, u32* slots,
                    unsigned long long* maxr, cudaStream_t st) {
  cudaMemsetAsync(maxr, 0, sizeof(unsigned long long), st);
  k_dec_z<<<V.k, ntt_threads(V.N), (size_t)V.N * 8, st>>>(V, ct, s_ntt, zbuf);
  k_dec_coef<<<grid_for(V.N, 128), 128, 0, st>>>(*V.host_args, V, zbuf, mbuf, maxr);
  k_dec_slots<<<1, ntt_threads(V.N), (size_t)V.N * 8, st>>>(V, mbuf, slots);
}

void launch_mask(const DevView& V, u64 seed, u64* ct, cudaStream_t st) {
  k_mask<<<1, 512, (size_t)V.N * 8, st>>>(V, seed, ct);
}

cudaError_t kernels_init(int N) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  // largest request: the plaintext generator at this N
  if ((size_t)optin < ptgen_smem(N) || (size_t)optin < (size_t)N * 12) return cudaErrorInvalidValue;
  // dynamic + static shared memory of a block must stay within the opt-in limit
  auto set = [&](const void* f) {
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, f);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (r != cudaSuccess && e == cudaSuccess) e = r;
  };
  set((const void*)k_ntt<true>);
  set((const void*)k_ntt<false>);
  set((const void*)k_ntt<true, true>);
  set((const void*)k_ptgen);
  set((const void*)k_valgen);
  set((const void*)k_mac<false>);
  set((const void*)k_mac<true>);
#define PEPSI_SET_MACQ(QB, RG)                         \
  set((const void*)k_mac_multi<QB, RG, 1, false>);     \
  set((const void*)k_mac_multi<QB, RG, 1, true>);      \
  set((const void*)k_mac_multi<QB, RG, 2, false>);     \
  set((const void*)k_mac_multi<QB, RG, 2, true>);
  PEPSI_SET_MACQ(2, 1)
  PEPSI_SET_MACQ(2, 2)
  PEPSI_SET_MACQ(3, 1)
  PEPSI_SET_MACQ(4, 1)
  PEPSI_SET_MACQ(4, 2)
#undef PEPSI_SET_MACQ
  set((const void*)k_relin_ntt<256>);
  set((const void*)k_relin_ntt<NTT_MAX_THREADS>);
  set((const void*)k_tensor_intt);
  set((const void*)k_axpy_intt);
  set((const void*)k_relin_axpy_intt<256>);
  set((const void*)k_relin_axpy_intt<NTT_MAX_THREADS>);
  set((const void*)k_encrypt);
  set((const void*)k_keygen_sntt);
  set((const void*)k_keygen_rlk);
  set((const void*)k_dec_z);
  set((const void*)k_dec_slots);
  set((const void*)k_mask);
  return e;
}

// ------------------------------------------------------ integer-pipe peak
// Throughput probe of the multiply forms the kernels above are built from:
// FORM 1, 32x32->64 wide multiply-add into a 64-bit sum (mad.wide.u32, the
// multiply-accumulate's operation); FORM 2, the wide product alone
// (mul.wide.u32); FORM 0, 32-bit multiply-add (mad.lo.u32).  Each thread runs
// 16 chains; the multiplier of chain i is the low word of chain i+5, so it
// changes every step and no product can be hoisted out of the loop.  The
// result is folded into *sink so nothing is dead code.
namespace {
template <int FORM>
__global__ void k_int_peak(int iters, u32 seed, u64* sink) {
  u64 a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = seed + threadIdx.x * 7 + i;
  const u32 m = seed | 1u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const u32 x = (u32)a[(i + 5) & 15];
      if (FORM == 1) {
        asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a[i]) : "r"(x), "r"(m));
      } else if (FORM == 2) {
        asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(a[i]) : "r"(x), "r"(m));
      } else {
        u32 l = (u32)a[i];
        asm volatile("mad.lo.u32 %0, %1, %2, %0;" : "+r"(l) : "r"(x), "r"(m));
        a[i] = (a[i] & 0xffffffff00000000ull) | l;
      }
    }
  }
  u64 acc = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) acc += a[i];
  if (acc == 0x123456789ull) *sink = acc;
}
}  // namespace

double measure_int_peak(int form) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  u64* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(u64)) != cudaSuccess) return 0;
  const int threads = 512, blocks = sms * 4, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    if (form == 1)
      k_int_peak<1><<<blocks, threads>>>(iters, 7u + rep, sink);
    else if (form == 2)
      k_int_peak<2><<<blocks, threads>>>(iters, 7u + rep, sink);
    else
      k_int_peak<0><<<blocks, threads>>>(iters, 7u + rep, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double ops = (double)blocks * threads * iters * 16;
    if (ms > 0) best = std::max(best, ops / (ms * 1e-3));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return best;
}
