// Block-cooperative negacyclic NTT on a shared-memory polynomial.
//
// Forward: natural-order coefficients in, values at psi^(2 brev(i)+1) in
// position i out (radix-2 Cooley-Tukey with twiddles psi^brev(m+i), the
// merged negacyclic form of Longa-Naehrig), Harvey's lazy butterflies.
// Inverse: Gentleman-Sande with psi^-brev(m+i), then the factor N^-1.
//
// The log2 N radix-2 stages run in phases of RR <= 3 consecutive stages.  The butterflies of stages [s0, s0+RR) only combine the 2^RR
// elements base + i * (N >> (s0+RR)), i < 2^RR, so a thread loads such a
// group into registers, runs the RR stages there and stores it back: one
// shared-memory round trip and one barrier per phase instead of per stage.
// Every thread of the block must call these (they contain __syncthreads);
// any block size works (threads loop over the groups).
//
// Shared-memory layout: logical element x lives at word nsw(x) = x ^ ((x >> 4)
// & 15).  Groups of a phase are read at element strides 2^k; with the XOR of
// the higher index bits into the low four, the 16 words a half-warp reads
// fall into 16 different 8-byte bank pairs for every such stride, and runs
// of consecutive elements stay conflict-free.  Callers filling or reading
// the array index it through nsw().
#pragma once
#include <type_traits>
#include "common.cuh"

__device__ __forceinline__ int nsw(int x) { return x ^ ((x >> 4) & 15); }

namespace nttd {

// Word types of the transforms: 64-bit words for the ciphertext primes, and
// 32-bit words for a modulus below 2^30 (the plaintext modulus t), where
// Shoup's product takes one 32x32 high product and two low ones.  A twiddle
// pair (w, floor(w 2^64 / q)) gives the 32-bit companion floor(w 2^32 / q)
// as its upper half.
__device__ __forceinline__ u64 lazy_mul(u64 x, u64 w, u64 ws, u64 q) { return shoup_lazy(x, w, ws, q); }
__device__ __forceinline__ u32 lazy_mul(u32 x, u32 w, u32 ws, u32 q) { return x * w - __umulhi(x, ws) * q; }
__device__ __forceinline__ void tw_split(const ulonglong2& t, u64& w, u64& ws) {
  w = t.x;
  ws = t.y;
}
__device__ __forceinline__ void tw_split(const ulonglong2& t, u32& w, u32& ws) {
  w = (u32)t.x;
  ws = (u32)(t.y >> 32);
}

// Forward stages [s0, s0 + RR) on one group of 2^RR elements held in
// registers, element i of the group at base + i * 2^(logN - s0 - RR).
// Twiddles come as (w, Shoup companion) pairs, one 16-byte load each.
// GROW: the butterfly's sum input is not reduced below 2q first, so values
// grow by 2q a stage (Shoup's product takes any 64-bit input and returns
// [0, 2q)): from [0, 4q) they stay below (4 + 2 log2 N) q <= 32 q, which fits
// 64 bits for q < 2^59; the transform's end reduces them (fwd_final_grow).
template <int RR, bool GROW = false>
__device__ __forceinline__ void fwd_group(u64 (&x)[1 << RR], int base, int logN, int s0, u64 q,
                                          const ulonglong2* __restrict__ tw) {
  constexpr int E = 1 << RR;
  const u64 q2 = 2 * q;
#pragma unroll
  for (int ss = 0; ss < RR; ++ss) {
    const int s = s0 + ss;
    const int half = 1 << (RR - 1 - ss);
    // base has zero bits where i * stride lands, so the twiddle index of
    // butterfly i splits into a group part and i >> (RR - ss): stage ss of
    // the phase needs only 2^ss distinct twiddles
    const int tbase = (1 << s) + (base >> (logN - s));
    ulonglong2 Wt[1 << (RR - 1)];
#pragma unroll
    for (int d = 0; d < (1 << ss); ++d) Wt[d] = __ldg(tw + tbase + d);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      if ((i & half) == 0) {
        const u64 W = Wt[i >> (RR - ss)].x, Ws = Wt[i >> (RR - ss)].y;
        u64 U = x[i];
        if constexpr (!GROW) U = U >= q2 ? U - q2 : U;
        const u64 T = shoup_lazy(x[i + half], W, Ws, q);
        x[i] = U + T;
        x[i + half] = U + q2 - T;
      }
    }
  }
}
// [0, 4q) -> [0, q)
template <int E>
__device__ __forceinline__ void fwd_final(u64 (&x)[E], u64 q) {
  const u64 q2 = 2 * q;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    u64 v = x[i];
    v = v >= q2 ? v - q2 : v;
    x[i] = v >= q ? v - q : v;
  }
}
// [0, 2^64) -> [0, q): one-word Barrett (floor(x m64 / 2^64) is short of
// floor(x / q) by at most 1), then one conditional subtraction.
template <int E>
__device__ __forceinline__ void fwd_final_grow(u64 (&x)[E], u64 q, u64 m64) {
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const u64 v = x[i] - __umul64hi(x[i], m64) * q;
    x[i] = v >= q ? v - q : v;
  }
}
// Inverse (Gentleman-Sande) stages s0 + RR - 1 down to s0 on one group.
template <int RR, class T>
__device__ __forceinline__ void inv_group(T (&x)[1 << RR], int base, int logN, int s0, T q,
                                          const ulonglong2* __restrict__ itw) {
  constexpr int E = 1 << RR;
  const T q2 = 2 * q;
#pragma unroll
  for (int ss = RR - 1; ss >= 0; --ss) {
    const int s = s0 + ss;
    const int half = 1 << (RR - 1 - ss);
    const int tbase = (1 << s) + (base >> (logN - s));
    ulonglong2 Wt[1 << (RR - 1)];
#pragma unroll
    for (int d = 0; d < (1 << ss); ++d) Wt[d] = __ldg(itw + tbase + d);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      if ((i & half) == 0) {
        T W, Ws;
        tw_split(Wt[i >> (RR - ss)], W, Ws);
        const T U = x[i], V = x[i + half];
        T S = U + V;
        S = S >= q2 ? S - q2 : S;
        x[i] = S;
        x[i + half] = lazy_mul((T)(U + q2 - V), W, Ws, q);
      }
    }
  }
}
// times N^-1, [0, 2q) -> [0, q)
template <int E, class T>
__device__ __forceinline__ void inv_final(T (&x)[E], T q, T ninv, T ninvs) {
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const T v = lazy_mul(x[i], ninv, ninvs, q);
    x[i] = v >= q ? v - q : v;
  }
}

// Stages 2, 1, 0 of the inverse on the radix-8 group at base, with the
// factor N^-1: the sums of stage 0 are multiplied by N^-1, the differences
// by the table's entry 0 (the stage-0 twiddle times N^-1) instead of by the
// twiddle, then every element is reduced to [0, q).  The same residues as
// inv_group<3> at s0 = 0 followed by inv_final, with half the products of
// the final scaling.
template <class T>
__device__ __forceinline__ void inv_group_last(T (&x)[8], int base, int logN, T q, const ulonglong2* __restrict__ itw,
                                               T ninv, T ninvs) {
  const T q2 = 2 * q;
#pragma unroll
  for (int ss = 2; ss >= 1; --ss) {
    const int half = 1 << (2 - ss);
    const int tbase = (1 << ss) + (base >> (logN - ss));
    ulonglong2 Wt[4];
#pragma unroll
    for (int d = 0; d < (1 << ss); ++d) Wt[d] = __ldg(itw + tbase + d);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if ((i & half) == 0) {
        T W, Ws;
        tw_split(Wt[i >> (3 - ss)], W, Ws);
        const T U = x[i], V = x[i + half];
        T S = U + V;
        S = S >= q2 ? S - q2 : S;
        x[i] = S;
        x[i + half] = lazy_mul((T)(U + q2 - V), W, Ws, q);
      }
    }
  }
  T Wn, Wns;
  tw_split(__ldg(itw), Wn, Wns);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T U = x[i], V = x[i + 4];
    T S = U + V;
    S = S >= q2 ? S - q2 : S;
    const T a = lazy_mul(S, ninv, ninvs, q), b = lazy_mul((T)(U + q2 - V), Wn, Wns, q);
    x[i] = a >= q ? a - q : a;
    x[i + 4] = b >= q ? b - q : b;
  }
}

template <int RR, bool GROW = false>
__device__ __forceinline__ void fwd_phase(u64* a, int N, int logN, int s0, u64 q, const ulonglong2* __restrict__ tw,
                                          bool last) {
  constexpr int E = 1 << RR;
  const int slog = logN - s0 - RR;  // log2 of the element stride inside a group
  const int groups = N >> RR;
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = ((g >> slog) << (slog + RR)) + (g & ((1 << slog) - 1));
    u64 x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = a[nsw(base + (i << slog))];
    fwd_group<RR, GROW>(x, base, logN, s0, q, tw);
    if (last) fwd_final<E>(x, q);
#pragma unroll
    for (int i = 0; i < E; ++i) a[nsw(base + (i << slog))] = x[i];
  }
}

template <int RR, class T>
__device__ __forceinline__ void inv_phase(T* a, int N, int logN, int s0, T q, const ulonglong2* __restrict__ itw,
                                          bool last, T ninv, T ninvs) {
  constexpr int E = 1 << RR;
  const int slog = logN - s0 - RR;
  const int groups = N >> RR;
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = ((g >> slog) << (slog + RR)) + (g & ((1 << slog) - 1));
    T x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = a[nsw(base + (i << slog))];
    inv_group<RR>(x, base, logN, s0, q, itw);
    if (last) inv_final<E>(x, q, ninv, ninvs);
#pragma unroll
    for (int i = 0; i < E; ++i) a[nsw(base + (i << slog))] = x[i];
  }
}

}  // namespace nttd

// a[0..N) in [0, 4q) on entry, [0, q) on exit.  Phases of three stages
// from stage 0, then the remaining one or two.
__device__ __forceinline__ void ntt_fwd_block(u64* a, int N, int logN, u64 q, const ulonglong2* __restrict__ tw) {
  int s0 = 0;
  for (; s0 + 3 <= logN; s0 += 3) {
    nttd::fwd_phase<3>(a, N, logN, s0, q, tw, s0 + 3 == logN);
    __syncthreads();
  }
  const int rem = logN - s0;
  if (rem == 2) nttd::fwd_phase<2>(a, N, logN, s0, q, tw, true);
  if (rem == 1) nttd::fwd_phase<1>(a, N, logN, s0, q, tw, true);
  if (rem) __syncthreads();
}

// a[0..N) in [0, 2q) on entry, [0, q) on exit.  The forward phases in
// reverse order: the remainder first, then three stages at a time.
template <class T>
__device__ __forceinline__ void ntt_inv_block(T* a, int N, int logN, T q, const ulonglong2* __restrict__ itw, T ninv,
                                              T ninvs) {
  const int rem = logN % 3;
  int s0 = logN - rem;
  if (rem == 2) nttd::inv_phase<2>(a, N, logN, s0, q, itw, s0 == 0, ninv, ninvs);
  if (rem == 1) nttd::inv_phase<1>(a, N, logN, s0, q, itw, s0 == 0, ninv, ninvs);
  if (rem) __syncthreads();
  for (s0 -= 3; s0 >= 0; s0 -= 3) {
    nttd::inv_phase<3>(a, N, logN, s0, q, itw, s0 == 0, ninv, ninvs);
    __syncthreads();
  }
}

__device__ __forceinline__ void ntt_fwd_view(u64* a, const DevView& V, int pi) {
  ntt_fwd_block(a, V.N, V.logN, V.pr[pi].q, V.twp + (size_t)pi * V.N);
}
__device__ __forceinline__ void ntt_inv_view(u64* a, const DevView& V, int pi) {
  const DevPrime P = V.pr[pi];
  ntt_inv_block(a, V.N, V.logN, P.q, V.itwp + (size_t)pi * V.N, P.ninv, P.ninvs);
}

// The same transforms with log2 N fixed at compile time: the phase bounds,
// strides and shift amounts become constants.
template <int LOGN>
__device__ __forceinline__ void ntt_fwd_fixed(u64* a, u64 q, const ulonglong2* __restrict__ tw) {
  constexpr int N = 1 << LOGN, REM = LOGN % 3;
#pragma unroll
  for (int s0 = 0; s0 + 3 <= LOGN; s0 += 3) {
    nttd::fwd_phase<3>(a, N, LOGN, s0, q, tw, s0 + 3 == LOGN);
    __syncthreads();
  }
  if constexpr (REM == 2) {
    nttd::fwd_phase<2>(a, N, LOGN, LOGN - 2, q, tw, true);
    __syncthreads();
  }
  if constexpr (REM == 1) {
    nttd::fwd_phase<1>(a, N, LOGN, LOGN - 1, q, tw, true);
    __syncthreads();
  }
}
template <int LOGN>
__device__ __forceinline__ void ntt_inv_fixed(u64* a, u64 q, const ulonglong2* __restrict__ itw, u64 ninv,
                                              u64 ninvs) {
  constexpr int N = 1 << LOGN, REM = LOGN % 3, TOP = LOGN - REM;
  if constexpr (REM == 2) {
    nttd::inv_phase<2>(a, N, LOGN, TOP, q, itw, TOP == 0, ninv, ninvs);
    __syncthreads();
  }
  if constexpr (REM == 1) {
    nttd::inv_phase<1>(a, N, LOGN, TOP, q, itw, TOP == 0, ninv, ninvs);
    __syncthreads();
  }
#pragma unroll
  for (int s0 = TOP - 3; s0 >= 0; s0 -= 3) {
    nttd::inv_phase<3>(a, N, LOGN, s0, q, itw, s0 == 0, ninv, ninvs);
    __syncthreads();
  }
}

// ntt_fwd_view / ntt_inv_view with the ring sizes of the workloads
// (N = 4096, 8192, 16384) compiled for their fixed size.
__device__ __forceinline__ void ntt_fwd_fast(u64* a, const DevView& V, int pi) {
  const ulonglong2* tw = V.twp + (size_t)pi * V.N;
  const u64 q = V.pr[pi].q;
  switch (V.logN) {
    case 12: ntt_fwd_fixed<12>(a, q, tw); break;
    case 13: ntt_fwd_fixed<13>(a, q, tw); break;
    case 14: ntt_fwd_fixed<14>(a, q, tw); break;
    default: ntt_fwd_block(a, V.N, V.logN, q, tw); break;
  }
}
__device__ __forceinline__ void ntt_inv_fast(u64* a, const DevView& V, int pi) {
  const ulonglong2* itw = V.itwp + (size_t)pi * V.N;
  const DevPrime P = V.pr[pi];
  switch (V.logN) {
    case 12: ntt_inv_fixed<12>(a, P.q, itw, P.ninv, P.ninvs); break;
    case 13: ntt_inv_fixed<13>(a, P.q, itw, P.ninv, P.ninvs); break;
    case 14: ntt_inv_fixed<14>(a, P.q, itw, P.ninv, P.ninvs); break;
    default: ntt_inv_block(a, V.N, V.logN, P.q, itw, P.ninv, P.ninvs); break;
  }
}

// Row accessors for the global-to-global transforms.  A functor with a
// pair(x, ...) member moves elements x and x + 1 (x even) together; the
// transforms use it for the groups of consecutive elements (the first group
// of the inverse, the last of the forward).  The row accessors do one
// 16-byte access when the row is 16-byte aligned (rows are whole multiples
// of N words from their base, so the test is uniform over a block) and two
// 8-byte accesses otherwise: caller buffers need only 8-byte alignment.
// Plain lambdas are used element by element.
template <class T, class = void>
struct has_pair : std::false_type {};
template <class T>
struct has_pair<T, std::void_t<decltype(&T::pair)>> : std::true_type {};
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
struct RowLd {
  const u64* p;
  bool v16;
  __device__ __forceinline__ explicit RowLd(const u64* row) : p(row), v16(aligned16(row)) {}
  __device__ __forceinline__ u64 operator()(int x) const { return p[x]; }
  __device__ __forceinline__ void pair(int x, u64& a, u64& b) const {
    if (v16) {
      const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(p + x);
      a = w.x;
      b = w.y;
    } else {
      a = p[x];
      b = p[x + 1];
    }
  }
};
struct RowSt {
  u64* p;
  bool v16;
  __device__ __forceinline__ explicit RowSt(u64* row) : p(row), v16(aligned16(row)) {}
  __device__ __forceinline__ void operator()(int x, u64 v) const { p[x] = v; }
  __device__ __forceinline__ void pair(int x, u64 a, u64 b) const {
    if (v16) {
      *reinterpret_cast<ulonglong2*>(p + x) = make_ulonglong2(a, b);
    } else {
      p[x] = a;
      p[x + 1] = b;
    }
  }
};
// the split operand format of the multiply-accumulate (shift s)
struct SplitSt {
  RowSt r;
  u64 s;
  __device__ __forceinline__ SplitSt(u64* row, u64 shift) : r(row), s(shift) {}
  __device__ __forceinline__ void operator()(int x, u64 v) const { r(x, to_split(v, s)); }
  __device__ __forceinline__ void pair(int x, u64 a, u64 b) const { r.pair(x, to_split(a, s), to_split(b, s)); }
};
// the split operand format plus the 32-bit sum of each word's halves
struct SplitSumSt {
  SplitSt w;
  u32* sum;
  __device__ __forceinline__ SplitSumSt(u64* row, u32* sums, u64 shift) : w(row, shift), sum(sums) {}
  __device__ __forceinline__ static u32 halves(u64 v) { return (u32)v + (u32)(v >> 32); }
  __device__ __forceinline__ void operator()(int x, u64 v) const {
    const u64 t = to_split(v, w.s);
    w.r(x, t);
    sum[x] = halves(t);
  }
  __device__ __forceinline__ void pair(int x, u64 a, u64 b) const {
    const u64 ta = to_split(a, w.s), tb = to_split(b, w.s);
    w.r.pair(x, ta, tb);
    sum[x] = halves(ta);
    sum[x + 1] = halves(tb);
  }
};
template <int E, class T, class Load>
__device__ __forceinline__ void load_run(T (&x)[E], const Load& ld, int base) {
  if constexpr (has_pair<Load>::value && E >= 2) {
#pragma unroll
    for (int i = 0; i < E; i += 2) ld.pair(base + i, x[i], x[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = ld(base + i);
  }
}
template <int E, class Store>
__device__ __forceinline__ void store_run(const u64 (&x)[E], const Store& st, int base) {
  if constexpr (has_pair<Store>::value && E >= 2) {
#pragma unroll
    for (int i = 0; i < E; i += 2) st.pair(base + i, x[i], x[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) st(base + i, x[i]);
  }
}

// Transforms from a row in global memory to a row in global memory through
// the shared-memory array a[].  The first three stages run on the registers
// of the global load and the last R stages (R = 1, 2 or 3, the rest after
// radix-8 phases) on those of the global store, so of the log2(N) stages
// only the middle ones take shared-memory phases (N = 8192: three instead
// of five).  The butterflies and their order are those of ntt_fwd_fixed /
// ntt_inv_fixed, so are the results.  ld(x) returns input element x (forward:
// in [0, 4q); inverse: in [0, 2q)); st(x, v) receives output element x,
// reduced.  Every read through ld happens before the first barrier and
// every st after the last, so input and output rows may alias.  Every
// thread of the block must call these.
// GROW (q < 2^59): butterflies without the reduction of their sum input,
// one Barrett reduction (m64 = floor(2^64 / q)) at the store; the same
// residues.
template <int LOGN, bool GROW, class Load, class Store>
__device__ __forceinline__ void ntt_fwd_fused(u64* a, const Load& ld, const Store& st, u64 q, u64 m64,
                                              const ulonglong2* __restrict__ tw) {
  constexpr int N = 1 << LOGN, R = (LOGN - 4) % 3 + 1, M = (LOGN - 3 - R) / 3, S8 = LOGN - 3;
  for (int g = threadIdx.x; g < (N >> 3); g += blockDim.x) {  // stages 0-2
    u64 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = ld(g + (i << S8));
    nttd::fwd_group<3, GROW>(x, g, LOGN, 0, q, tw);
#pragma unroll
    for (int i = 0; i < 8; ++i) a[nsw(g + (i << S8))] = x[i];
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < M; ++m) {
    nttd::fwd_phase<3, GROW>(a, N, LOGN, 3 + 3 * m, q, tw, false);
    __syncthreads();
  }
  for (int g = threadIdx.x; g < (N >> R); g += blockDim.x) {  // stages LOGN-R .. LOGN-1
    const int base = g << R;
    u64 x[1 << R];
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) x[i] = a[nsw(base + i)];
    nttd::fwd_group<R, GROW>(x, base, LOGN, LOGN - R, q, tw);
    if constexpr (GROW)
      nttd::fwd_final_grow<1 << R>(x, q, m64);
    else
      nttd::fwd_final<1 << R>(x, q);
    store_run<1 << R>(x, st, base);
  }
}
template <int LOGN, class T, class Load, class Store>
__device__ __forceinline__ void ntt_inv_fused(T* a, const Load& ld, const Store& st, T q,
                                              const ulonglong2* __restrict__ itw, T ninv, T ninvs) {
  constexpr int N = 1 << LOGN, R = (LOGN - 4) % 3 + 1, M = (LOGN - 3 - R) / 3, S8 = LOGN - 3;
  for (int g = threadIdx.x; g < (N >> R); g += blockDim.x) {  // stages LOGN-1 .. LOGN-R
    const int base = g << R;
    T x[1 << R];
    load_run<1 << R>(x, ld, base);
    nttd::inv_group<R>(x, base, LOGN, LOGN - R, q, itw);
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) a[nsw(base + i)] = x[i];
  }
  __syncthreads();
#pragma unroll
  for (int m = M - 1; m >= 0; --m) {
    nttd::inv_phase<3>(a, N, LOGN, 3 + 3 * m, q, itw, false, ninv, ninvs);
    __syncthreads();
  }
  for (int g = threadIdx.x; g < (N >> 3); g += blockDim.x) {  // stages 2-0 and N^-1
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = a[nsw(g + (i << S8))];
    nttd::inv_group_last(x, g, LOGN, q, itw, ninv, ninvs);
#pragma unroll
    for (int i = 0; i < 8; ++i) st(g + (i << S8), x[i]);
  }
}

// Global-to-global transforms of row pi with the fused forms for the ring
// sizes of the workloads (N = 4096, 8192, 16384), else load, block
// transform and store.
template <class Load, class Store>
__device__ __forceinline__ void ntt_fwd_gg(u64* a, const Load& ld, const Store& st, const DevView& V, int pi) {
  const ulonglong2* tw = V.twp + (size_t)pi * V.N;
  const DevPrime P = V.pr[pi];
  const u64 q = P.q;
  // values reach (4 + 2 log2 N) q <= 32 q without per-stage reduction
  const bool grow = q < (1ull << 59);
  switch (V.logN * 2 + (grow ? 1 : 0)) {
    case 12 * 2: ntt_fwd_fused<12, false>(a, ld, st, q, P.m64, tw); return;
    case 12 * 2 + 1: ntt_fwd_fused<12, true>(a, ld, st, q, P.m64, tw); return;
    case 13 * 2: ntt_fwd_fused<13, false>(a, ld, st, q, P.m64, tw); return;
    case 13 * 2 + 1: ntt_fwd_fused<13, true>(a, ld, st, q, P.m64, tw); return;
    case 14 * 2: ntt_fwd_fused<14, false>(a, ld, st, q, P.m64, tw); return;
    case 14 * 2 + 1: ntt_fwd_fused<14, true>(a, ld, st, q, P.m64, tw); return;
    default: break;
  }
  for (int x = threadIdx.x; x < V.N; x += blockDim.x) a[nsw(x)] = ld(x);
  __syncthreads();
  ntt_fwd_block(a, V.N, V.logN, q, tw);
  for (int x = threadIdx.x; x < V.N; x += blockDim.x) st(x, a[nsw(x)]);
}
template <class Load, class Store>
__device__ __forceinline__ void ntt_inv_gg(u64* a, const Load& ld, const Store& st, const DevView& V, int pi) {
  const ulonglong2* itw = V.itwp + (size_t)pi * V.N;
  const DevPrime P = V.pr[pi];
  switch (V.logN) {
    case 12: ntt_inv_fused<12>(a, ld, st, P.q, itw, P.ninv, P.ninvs); return;
    case 13: ntt_inv_fused<13>(a, ld, st, P.q, itw, P.ninv, P.ninvs); return;
    case 14: ntt_inv_fused<14>(a, ld, st, P.q, itw, P.ninv, P.ninvs); return;
    default: break;
  }
  for (int x = threadIdx.x; x < V.N; x += blockDim.x) a[nsw(x)] = ld(x);
  __syncthreads();
  ntt_inv_block(a, V.N, V.logN, P.q, itw, P.ninv, P.ninvs);
  for (int x = threadIdx.x; x < V.N; x += blockDim.x) st(x, a[nsw(x)]);
}

// ntt_inv_gg for a modulus q_pi below 2^30 (the plaintext modulus) in 32-bit
// words: a[] holds N 32-bit words, ld(x) returns element x in [0, 2q) as
// u32, st(x, v) receives it reduced.  The same residues as ntt_inv_gg.
template <class Load, class Store>
__device__ __forceinline__ void ntt_inv_gg_small(u32* a, const Load& ld, const Store& st, const DevView& V, int pi) {
  const ulonglong2* itw = V.itwp + (size_t)pi * V.N;
  const DevPrime P = V.pr[pi];
  const u32 q = (u32)P.q, ninv = (u32)P.ninv, ninvs = (u32)(P.ninvs >> 32);
  switch (V.logN) {
    case 12: ntt_inv_fused<12>(a, ld, st, q, itw, ninv, ninvs); return;
    case 13: ntt_inv_fused<13>(a, ld, st, q, itw, ninv, ninvs); return;
    case 14: ntt_inv_fused<14>(a, ld, st, q, itw, ninv, ninvs); return;
    default: break;
  }
  for (int x = threadIdx.x; x < V.N; x += blockDim.x) a[nsw(x)] = ld(x);
  __syncthreads();
  ntt_inv_block(a, V.N, V.logN, q, itw, ninv, ninvs);
  for (int x = threadIdx.x; x < V.N; x += blockDim.x) st(x, a[nsw(x)]);
}
