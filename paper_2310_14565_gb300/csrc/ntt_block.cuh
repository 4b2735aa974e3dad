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
#include "common.cuh"

__device__ __forceinline__ int nsw(int x) { return x ^ ((x >> 4) & 15); }

namespace nttd {

// Phase sizes for log2 N stages: 3-stage phases, then the remainder.
__device__ __forceinline__ int phase_plan(int logN, int* r) {
  int n = 0, rest = logN;
  while (rest >= 3) {
    r[n++] = 3;
    rest -= 3;
  }
  if (rest) r[n++] = rest;
  return n;
}

template <int RR>
__device__ __forceinline__ void fwd_phase(u64* a, int N, int logN, int s0, u64 q, const u64* __restrict__ tw,
                                          const u64* __restrict__ tws, bool last) {
  constexpr int E = 1 << RR;
  const int slog = logN - s0 - RR;  // log2 of the element stride inside a group
  const int groups = N >> RR;
  const u64 q2 = 2 * q;
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = ((g >> slog) << (slog + RR)) + (g & ((1 << slog) - 1));
    u64 x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = a[nsw(base + (i << slog))];
#pragma unroll
    for (int ss = 0; ss < RR; ++ss) {
      const int s = s0 + ss;
      const int half = 1 << (RR - 1 - ss);
      // base has zero bits where i * stride lands, so the twiddle index of
      // butterfly i splits into a group part and i >> (RR - ss): stage ss of
      // the phase needs only 2^ss distinct twiddles
      const int tbase = (1 << s) + (base >> (logN - s));
      u64 Wt[1 << (RR - 1)], Wst[1 << (RR - 1)];
#pragma unroll
      for (int d = 0; d < (1 << ss); ++d) {
        Wt[d] = __ldg(tw + tbase + d);
        Wst[d] = __ldg(tws + tbase + d);
      }
#pragma unroll
      for (int i = 0; i < E; ++i) {
        if ((i & half) == 0) {
          const u64 W = Wt[i >> (RR - ss)], Ws = Wst[i >> (RR - ss)];
          u64 U = x[i];
          U = U >= q2 ? U - q2 : U;
          const u64 T = shoup_lazy(x[i + half], W, Ws, q);
          x[i] = U + T;
          x[i + half] = U + q2 - T;
        }
      }
    }
    if (last) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        u64 v = x[i];
        v = v >= q2 ? v - q2 : v;
        x[i] = v >= q ? v - q : v;
      }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) a[nsw(base + (i << slog))] = x[i];
  }
}

template <int RR>
__device__ __forceinline__ void inv_phase(u64* a, int N, int logN, int s0, u64 q, const u64* __restrict__ itw,
                                          const u64* __restrict__ itws, bool last, u64 ninv, u64 ninvs) {
  constexpr int E = 1 << RR;
  const int slog = logN - s0 - RR;
  const int groups = N >> RR;
  const u64 q2 = 2 * q;
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int base = ((g >> slog) << (slog + RR)) + (g & ((1 << slog) - 1));
    u64 x[E];
#pragma unroll
    for (int i = 0; i < E; ++i) x[i] = a[nsw(base + (i << slog))];
#pragma unroll
    for (int ss = RR - 1; ss >= 0; --ss) {
      const int s = s0 + ss;
      const int half = 1 << (RR - 1 - ss);
      const int tbase = (1 << s) + (base >> (logN - s));
      u64 Wt[1 << (RR - 1)], Wst[1 << (RR - 1)];
#pragma unroll
      for (int d = 0; d < (1 << ss); ++d) {
        Wt[d] = __ldg(itw + tbase + d);
        Wst[d] = __ldg(itws + tbase + d);
      }
#pragma unroll
      for (int i = 0; i < E; ++i) {
        if ((i & half) == 0) {
          const u64 W = Wt[i >> (RR - ss)], Ws = Wst[i >> (RR - ss)];
          const u64 U = x[i], V = x[i + half];
          u64 S = U + V;
          S = S >= q2 ? S - q2 : S;
          x[i] = S;
          x[i + half] = shoup_lazy(U + q2 - V, W, Ws, q);
        }
      }
    }
    if (last) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const u64 v = shoup_lazy(x[i], ninv, ninvs, q);
        x[i] = v >= q ? v - q : v;
      }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) a[nsw(base + (i << slog))] = x[i];
  }
}

}  // namespace nttd

// a[0..N) in [0, 4q) on entry, [0, q) on exit.
__device__ __forceinline__ void ntt_fwd_block(u64* a, int N, int logN, u64 q, const u64* __restrict__ tw,
                                              const u64* __restrict__ tws) {
  int r[16];
  const int np = nttd::phase_plan(logN, r);
  int s0 = 0;
  for (int p = 0; p < np; ++p) {
    const bool last = p == np - 1;
    switch (r[p]) {
      case 3: nttd::fwd_phase<3>(a, N, logN, s0, q, tw, tws, last); break;
      case 2: nttd::fwd_phase<2>(a, N, logN, s0, q, tw, tws, last); break;
      default: nttd::fwd_phase<1>(a, N, logN, s0, q, tw, tws, last); break;
    }
    s0 += r[p];
    __syncthreads();
  }
}

// a[0..N) in [0, 2q) on entry, [0, q) on exit.
__device__ __forceinline__ void ntt_inv_block(u64* a, int N, int logN, u64 q, const u64* __restrict__ itw,
                                              const u64* __restrict__ itws, u64 ninv, u64 ninvs) {
  int r[16];
  const int np = nttd::phase_plan(logN, r);
  int s0 = logN;
  for (int p = np - 1; p >= 0; --p) {
    s0 -= r[p];
    const bool last = p == 0;
    switch (r[p]) {
      case 3: nttd::inv_phase<3>(a, N, logN, s0, q, itw, itws, last, ninv, ninvs); break;
      case 2: nttd::inv_phase<2>(a, N, logN, s0, q, itw, itws, last, ninv, ninvs); break;
      default: nttd::inv_phase<1>(a, N, logN, s0, q, itw, itws, last, ninv, ninvs); break;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void ntt_fwd_view(u64* a, const DevView& V, int pi) {
  const size_t off = (size_t)pi * V.N;
  ntt_fwd_block(a, V.N, V.logN, V.pr[pi].q, V.tw + off, V.tws + off);
}
__device__ __forceinline__ void ntt_inv_view(u64* a, const DevView& V, int pi) {
  const size_t off = (size_t)pi * V.N;
  const DevPrime P = V.pr[pi];
  ntt_inv_block(a, V.N, V.logN, P.q, V.itw + off, V.itws + off, P.ninv, P.ninvs);
}
