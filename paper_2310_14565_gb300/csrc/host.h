// Host-side parameter derivation and hashing of the PEPSI library.
#pragma once
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace hostmath {

typedef unsigned __int128 u128;

u64 mulmod(u64 a, u64 b, u64 m);
u64 powmod(u64 b, u64 e, u64 m);
u64 invmod(u64 a, u64 m);  // extended Euclid, m need not be prime
bool is_prime(u64 n);
// largest prime q < 2^bits with q = 1 mod 2N, not in taken
u64 find_prime(int bits, u32 N, const std::vector<u64>& taken);
// smallest w with w^N = -1 mod q
u64 min_root(u64 q, u32 N);
u64 shoup_of(u64 w, u64 q);
DevPrime make_prime(u64 q, u32 N);
// twiddles psi^brev(i) (fwd) and psi^-brev(i) (inv) with Shoup companions
void twiddles(u64 q, u64 psi, u32 N, u64* tw, u64* tws, u64* itw, u64* itws);
// constants of the exact RNS conversions
void rns_constants(const std::vector<u64>& Qp, const std::vector<u64>& Bp, u64 t, RnsConst* rc);
// round(Q v / t) mod q_i for v in [0, t)
void delta(const std::vector<u64>& Qp, u64 t, u64 v, u64* out);

// Eq. 1
u32 code_length(u32 lambda_bar, u32 h);
// Eq. 1 for any ell (binary search), 0 for unsupported arguments
u64 code_length_any(u32 lambda_bar, u32 h);
// Table 3: (log2 N, log2 q) for Hamming weight h in 1..64
bool table3(u32 h, u32* log2n, u32* log2q);
u64 binom_sat(u64 n, u64 r);
// server bin bound: the paper's values for its (n, b) pairs, else the
// smallest mu with b * P[Binomial(3n, 1/b) > mu] <= 2^-40
u32 mu_rule(u64 n, u32 b);

// hashing (Section 3.3): x -> x_L and its three bins
struct Hasher {
  u64 k0, k1, k2, k3;
  u32 lambda_bar, logb;
  Hasher(u64 hash_key, u32 lambda_bar, u32 logb);
  void operator()(u64 x, u64* xL, u32 bins[3]) const;
};
// client cuckoo hashing without stash into bins of gamma slots: table[bin*gamma + slot],
// where[u] = bin*gamma + slot; returns 0 or PEPSI_E_CUCKOO_FAIL
int cuckoo(const Hasher& H, const u64* items, size_t m, u32 gamma, std::vector<u64>& table,
           std::vector<int32_t>& where);
// Server simple hashing: T[mu][b] (x_L or PEPSI_DUMMY); with values, also
// V[mu][b], the value of the item stored at each (layer, bin), 0 for
// dummies.  Returns 0 or PEPSI_E_BIN_OVERFLOW.
int simple_hash(const Hasher& H, const u64* items, size_t n, u32 mu, std::vector<u64>& T, u32* max_load,
                const uint32_t* values = nullptr, std::vector<uint32_t>* V = nullptr);

}  // namespace hostmath
