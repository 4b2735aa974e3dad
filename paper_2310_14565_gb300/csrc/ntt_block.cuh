// Block-cooperative negacyclic NTT on a shared-memory polynomial.
//
// Forward: natural-order coefficients in, values at psi^(2 brev(i)+1) in
// position i out (radix-2 Cooley-Tukey with twiddles psi^brev(m+i), the
// merged negacyclic form of Longa-Naehrig), Harvey's lazy butterflies.
// Inverse: Gentleman-Sande with psi^-brev(m+i), then the factor N^-1.
// Every thread of the block must call these (they contain __syncthreads).
#pragma once
#include "common.cuh"

// a[0..N) in [0, 4q) on entry, [0, q) on exit.
__device__ __forceinline__ void ntt_fwd_block(u64* a, int N, int logN, u64 q, const u64* __restrict__ tw,
                                              const u64* __restrict__ tws) {
  const u64 q2 = 2 * q;
  const int half = N >> 1;
  for (int s = 0; s < logN; ++s) {
    const int m = 1 << s;
    const int lenlog = logN - 1 - s;
    const int len = 1 << lenlog;
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      const int i = b >> lenlog;
      const int j = (i << (lenlog + 1)) + (b & (len - 1));
      const u64 W = __ldg(tw + m + i), Ws = __ldg(tws + m + i);
      u64 U = a[j];
      U = U >= q2 ? U - q2 : U;
      const u64 T = shoup_lazy(a[j + len], W, Ws, q);
      a[j] = U + T;
      a[j + len] = U + q2 - T;
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    u64 v = a[x];
    v = v >= q2 ? v - q2 : v;
    a[x] = v >= q ? v - q : v;
  }
  __syncthreads();
}

// a[0..N) in [0, 2q) on entry, [0, q) on exit.
__device__ __forceinline__ void ntt_inv_block(u64* a, int N, int logN, u64 q, const u64* __restrict__ itw,
                                              const u64* __restrict__ itws, u64 ninv, u64 ninvs) {
  const u64 q2 = 2 * q;
  const int half = N >> 1;
  for (int s = logN - 1; s >= 0; --s) {
    const int m = 1 << s;
    const int lenlog = logN - 1 - s;
    const int len = 1 << lenlog;
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      const int i = b >> lenlog;
      const int j = (i << (lenlog + 1)) + (b & (len - 1));
      const u64 W = __ldg(itw + m + i), Ws = __ldg(itws + m + i);
      const u64 U = a[j], V = a[j + len];
      u64 S = U + V;
      S = S >= q2 ? S - q2 : S;
      a[j] = S;
      a[j + len] = shoup_lazy(U + q2 - V, W, Ws, q);
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    u64 v = shoup_lazy(a[x], ninv, ninvs, q);
    a[x] = v >= q ? v - q : v;
  }
  __syncthreads();
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
