// Host-side parameter derivation and hashing of the PEPSI library:
// prime search, roots of unity, NTT tables, the RNS conversion constants
// (computed from residues only), Eq. 1, the server bin bound, and the
// client / server hashing of Section 3.3 and App. Alg 7.
#include "host.h"

#include "pepsi.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <thread>

namespace hostmath {

u64 mulmod(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
u64 powmod(u64 b, u64 e, u64 m) {
  u64 r = 1 % m;
  b %= m;
  for (; e; e >>= 1) {
    if (e & 1) r = mulmod(r, b, m);
    b = mulmod(b, b, m);
  }
  return r;
}
u64 invmod(u64 a, u64 m) {
  // extended Euclid on signed 128-bit values
  __int128 r0 = m, r1 = a % m, s0 = 0, s1 = 1;
  while (r1) {
    __int128 qq = r0 / r1, tmp = r0 - qq * r1;
    r0 = r1;
    r1 = tmp;
    tmp = s0 - qq * s1;
    s0 = s1;
    s1 = tmp;
  }
  if (s0 < 0) s0 += m;
  return (u64)s0;
}

// Miller-Rabin with the seven bases of Jaeschke / Sinclair, exact below 2^64.
bool is_prime(u64 n) {
  if (n < 2) return false;
  for (u64 p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull}) {
    if (n % p == 0) return n == p;
  }
  u64 d = n - 1;
  int s = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++s;
  }
  for (u64 a : {2ull, 325ull, 9375ull, 28178ull, 450775ull, 9780504ull, 1795265022ull}) {
    u64 x = powmod(a % n, d, n);
    if (a % n == 0 || x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int r = 1; r < s && witness; ++r) {
      x = mulmod(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

u64 find_prime(int bits, u32 N, const std::vector<u64>& taken) {
  const u64 step = 2ull * N;
  if (bits > 62 || (1ull << bits) <= step) return 0;
  for (u64 q = (1ull << bits) - step + 1; q > step; q -= step) {
    if (std::find(taken.begin(), taken.end(), q) != taken.end()) continue;
    if (is_prime(q)) return q;
  }
  return 0;
}

u64 min_root(u64 q, u32 N) {
  const u64 e = (q - 1) / (2ull * N);
  u64 w = 0;
  for (u64 g = 2; g < q && !w; ++g) {
    u64 c = powmod(g, e, q);
    if (powmod(c, N, q) == q - 1) w = c;
  }
  if (!w) return 0;
  // every primitive 2N-th root is w^(2j+1)
  u64 best = w, x = w, w2 = mulmod(w, w, q);
  for (u32 j = 1; j < N; ++j) {
    x = mulmod(x, w2, q);
    best = std::min(best, x);
  }
  return best;
}

u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

DevPrime make_prime(u64 q, u32 N) {
  DevPrime p;
  p.q = q;
  p.ninv = invmod(N % q, q);
  p.ninvs = shoup_of(p.ninv, q);
  const int bits = 64 - __builtin_clzll(q);
  p.split = (u64)((bits + 1) / 2);
  p.nbits = (u64)bits;
  p.mu = (u64)(((u128)1 << (bits + 63)) / q);  // < 2^64: q > 2^(bits-1)
  p.m64 = (u64)(((u128)1 << 64) / q);
  p.c64 = (u64)(((u128)1 << 64) % q);
  p.c64s = shoup_of(p.c64, q);
  return p;
}

static u32 bitrev(u32 x, u32 bits) {
  u32 r = 0;
  for (u32 i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

void twiddles(u64 q, u64 psi, u32 N, u64* tw, u64* tws, u64* itw, u64* itws) {
  u32 lg = 0;
  while ((1u << lg) < N) ++lg;
  std::vector<u64> pw(N), ipw(N);
  const u64 ipsi = invmod(psi, q);
  pw[0] = ipw[0] = 1;
  for (u32 i = 1; i < N; ++i) {
    pw[i] = mulmod(pw[i - 1], psi, q);
    ipw[i] = mulmod(ipw[i - 1], ipsi, q);
  }
  for (u32 i = 0; i < N; ++i) {
    const u32 r = bitrev(i, lg);
    tw[i] = pw[r];
    tws[i] = shoup_of(tw[i], q);
    itw[i] = ipw[r];
    itws[i] = shoup_of(itw[i], q);
  }
  // entry 0 is not a stage twiddle (stage s uses [2^s, 2^(s+1))): the
  // inverse table keeps there its stage-0 twiddle times N^-1, which the last
  // inverse stage applies to its difference outputs
  if (N > 1) {
    itw[0] = mulmod(itw[1], invmod(N % q, q), q);
    itws[0] = shoup_of(itw[0], q);
  }
}

// Garner digits of the integer whose residues are x over primes p.
static std::vector<u64> garner(const std::vector<u64>& x, const std::vector<u64>& p) {
  std::vector<u64> v(p.size());
  for (size_t i = 0; i < p.size(); ++i) {
    u64 a = x[i] % p[i];
    for (size_t j = 0; j < i; ++j) {
      a = (a + p[i] - v[j] % p[i]) % p[i];
      a = mulmod(a, invmod(p[j] % p[i], p[i]), p[i]);
    }
    v[i] = a;
  }
  return v;
}

void rns_constants(const std::vector<u64>& Q, const std::vector<u64>& B, u64 t, RnsConst* rc) {
  const size_t k = Q.size(), kb = B.size();
  *rc = RnsConst{};
  for (size_t i = 0; i < k; ++i)
    for (size_t j = 0; j < i; ++j) {
      rc->cq[i][j] = invmod(Q[j] % Q[i], Q[i]);
      rc->cqs[i][j] = shoup_of(rc->cq[i][j], Q[i]);
    }
  for (size_t i = 0; i < kb; ++i)
    for (size_t j = 0; j < i; ++j) {
      rc->cb[i][j] = invmod(B[j] % B[i], B[i]);
      rc->cbs[i][j] = shoup_of(rc->cb[i][j], B[i]);
    }
  auto prod_mod = [](const std::vector<u64>& ps, size_t upto, u64 m) {
    u64 r = 1 % m;
    for (size_t l = 0; l < upto; ++l) r = mulmod(r, ps[l] % m, m);
    return r;
  };
  for (size_t j = 0; j < kb; ++j) {
    for (size_t l = 0; l < k; ++l) {
      rc->qb[j][l] = Q[l] % B[j];
      rc->qbs[j][l] = shoup_of(rc->qb[j][l], B[j]);
    }
    rc->qmodb[j] = prod_mod(Q, k, B[j]);
    const u64 inv2 = invmod(2, B[j]);
    rc->qhalf_b[j] = mulmod((rc->qmodb[j] + B[j] - 1) % B[j], inv2, B[j]);
    rc->qinv_b[j] = invmod(rc->qmodb[j], B[j]);
    rc->qinv_bs[j] = shoup_of(rc->qinv_b[j], B[j]);
    rc->t_b[j] = t % B[j];
    rc->t_bs[j] = shoup_of(rc->t_b[j], B[j]);
  }
  // (Q-1)/2 = -1/2 mod q_i, i.e. (q_i - 1)/2; its Garner digits over Q
  std::vector<u64> qh(k);
  for (size_t i = 0; i < k; ++i) {
    qh[i] = (Q[i] - 1) / 2;
    rc->qhalf_q[i] = qh[i];
    rc->t_q[i] = t % Q[i];
    rc->t_qs[i] = shoup_of(rc->t_q[i], Q[i]);
  }
  std::vector<u64> d = garner(qh, Q);
  for (size_t i = 0; i < k; ++i) rc->qhalf_dig[i] = d[i];
  std::vector<u64> bh(kb);
  for (size_t j = 0; j < kb; ++j) bh[j] = (B[j] - 1) / 2;
  d = garner(bh, B);
  for (size_t j = 0; j < kb; ++j) rc->bhalf_dig[j] = d[j];
  for (size_t i = 0; i < k; ++i) {
    for (size_t j = 0; j < kb; ++j) {
      rc->bq[i][j] = B[j] % Q[i];
      rc->bqs[i][j] = shoup_of(rc->bq[i][j], Q[i]);
    }
    rc->bmodq[i] = prod_mod(B, kb, Q[i]);
  }
  // decryption / encoding
  double acc = 1.0;
  for (size_t l = 0; l < k; ++l) {
    rc->pq_t[l] = prod_mod(Q, l, t);
    rc->pq_d[l] = acc;
    acc *= (double)Q[l];
  }
  const u64 qmt = prod_mod(Q, k, t);
  rc->qmt = qmt;
  rc->qinv_t = invmod(qmt, t);
  rc->qhalf_t = mulmod((qmt + t - 1) % t, invmod(2, t), t);
  for (size_t i = 0; i < k; ++i) {
    // floor(Q/t) = (Q - (Q mod t)) / t = -(Q mod t) * t^-1 mod q_i
    rc->qdt_q[i] = mulmod((Q[i] - qmt % Q[i]) % Q[i], invmod(t % Q[i], Q[i]), Q[i]);
    rc->qdt_qs[i] = shoup_of(rc->qdt_q[i], Q[i]);
  }
}

void delta(const std::vector<u64>& Q, u64 t, u64 v, u64* out) {
  u64 qmt = 1 % t;
  for (u64 q : Q) qmt = mulmod(qmt, q % t, t);
  const u64 frac = (u64)(((u128)qmt * v + (t - 1) / 2) / t);
  for (size_t i = 0; i < Q.size(); ++i) {
    const u64 qdt = mulmod((Q[i] - qmt % Q[i]) % Q[i], invmod(t % Q[i], Q[i]), Q[i]);
    out[i] = (mulmod(qdt, v % Q[i], Q[i]) + frac % Q[i]) % Q[i];
  }
}

u64 binom_sat(u64 n, u64 r) {
  if (r > n) return 0;
  u128 v = 1;
  for (u64 i = 1; i <= r; ++i) {
    v = v * (n - r + i) / i;
    if (v >> 63) return 1ull << 63;
  }
  return (u64)v;
}

u32 code_length(u32 lambda_bar, u32 h) {
  if (h == 0 || lambda_bar >= 63) return 0;
  for (u32 ell = h; ell < (1u << 20); ++ell)
    if (binom_sat(ell, h) >= (1ull << lambda_bar)) return ell;
  return 0;
}

u32 mu_rule(u64 n, u32 b) {
  static const std::map<std::pair<u64, u32>, u32> paper = {
      {{1ull << 20, 8192}, 526},   {{1ull << 24, 8192}, 6710}, {{1ull << 28, 8192}, 100565},
      {{1ull << 18, 16384}, 100},  {{1ull << 20, 16384}, 296}, {{1ull << 22, 16384}, 976},
      {{1ull << 24, 16384}, 3487}, {{1ull << 28, 16384}, 50812}};
  auto it = paper.find({n, b});
  if (it != paper.end()) return it->second;
  // tail P[X > mu] of Binomial(3n, 1/b), summed from the log-pmf
  const long double trials = 3.0L * n, p = 1.0L / b;
  const long double target = std::ldexp(1.0L, -40) / b;
  auto logpmf = [&](long double x) {
    return std::lgamma(trials + 1) - std::lgamma(x + 1) - std::lgamma(trials - x + 1) + x * std::log(p) +
           (trials - x) * std::log1p(-p);
  };
  u32 mu = (u32)std::max<long double>(1.0L, std::floor(trials * p));
  for (;; ++mu) {
    long double tail = 0;
    for (u64 x = mu + 1; x <= (u64)trials; ++x) {
      const long double term = std::exp(logpmf((long double)x));
      tail += term;
      if (term < tail * 1e-20L) break;
    }
    if (tail <= target) return mu;
  }
}

Hasher::Hasher(u64 hash_key, u32 lb, u32 lgb) : lambda_bar(lb), logb(lgb) {
  // K_i = i-th output of SplitMix64 seeded with hash_key
  k0 = mix64(hash_key + 1 * PEPSI_GOLDEN);
  k1 = mix64(hash_key + 2 * PEPSI_GOLDEN);
  k2 = mix64(hash_key + 3 * PEPSI_GOLDEN);
  k3 = mix64(hash_key + 4 * PEPSI_GOLDEN);
}
void Hasher::operator()(u64 x, u64* xL, u32 bins[3]) const {
  const u32 lam = lambda_bar + logb;
  u64 hx = mix64(x ^ k0);
  if (lam < 64) hx &= (1ull << lam) - 1;
  const u64 xh = hx >> lambda_bar;
  *xL = hx & ((1ull << lambda_bar) - 1);
  const u64 bm = (1ull << logb) - 1;
  bins[0] = (u32)(xh ^ (mix64(*xL ^ k1) & bm));
  bins[1] = (u32)(xh ^ (mix64(*xL ^ k2) & bm));
  bins[2] = (u32)(xh ^ (mix64(*xL ^ k3) & bm));
}

// Cuckoo hashing into bins of gamma slots (Section 4, the client's maximum
// bin load): items in input order take the first free slot of their current
// bin, starting at H_1; in a full bin the occupant of slot (evictions of this
// insertion so far) mod gamma is evicted and moves to its next hash function.
int cuckoo(const Hasher& H, const u64* items, size_t m, u32 gamma, std::vector<u64>& table,
           std::vector<int32_t>& where) {
  const u32 b = 1u << H.logb;
  if (gamma < 1) return PEPSI_E_PARAM;
  const size_t cells = (size_t)b * gamma;
  std::vector<int64_t> slot(cells, -1);  // item index, [bin][slot]
  std::vector<uint8_t> slot_h(cells, 0);
  std::vector<u32> load(b, 0);
  std::vector<u64> xl(m);
  std::vector<u32> bins(3 * m);
  for (size_t u = 0; u < m; ++u) H(items[u], &xl[u], &bins[3 * u]);
  for (size_t u = 0; u < m; ++u) {
    int64_t cur = (int64_t)u;
    int hidx = 0;
    for (int evictions = 0;; ++evictions) {
      const u32 bin = bins[3 * cur + hidx];
      if (load[bin] < gamma) {
        const size_t c = (size_t)bin * gamma + load[bin]++;
        slot[c] = cur;
        slot_h[c] = (uint8_t)hidx;
        break;
      }
      if (evictions >= 1000) return PEPSI_E_CUCKOO_FAIL;
      const size_t c = (size_t)bin * gamma + (u32)evictions % gamma;
      std::swap(slot[c], cur);
      int old_h = slot_h[c];
      slot_h[c] = (uint8_t)hidx;
      hidx = (old_h + 1) % 3;
    }
  }
  table.assign(cells, PEPSI_DUMMY);
  where.assign(m, -1);
  for (size_t i = 0; i < cells; ++i)
    if (slot[i] >= 0) {
      table[i] = xl[slot[i]];
      where[slot[i]] = (int32_t)i;
    }
  return 0;
}

// run f(lo, hi) over [0, count) split across the host's cores
template <class F>
static void parallel_ranges(size_t count, F f) {
  const size_t nt = std::max<size_t>(1, std::min<size_t>(std::thread::hardware_concurrency(), 64));
  if (nt == 1 || count < 4096) {
    f((size_t)0, count);
    return;
  }
  std::vector<std::thread> th;
  for (size_t t = 0; t < nt; ++t) {
    const size_t lo = count * t / nt, hi = count * (t + 1) / nt;
    th.emplace_back([=] { f(lo, hi); });
  }
  for (auto& x : th) x.join();
}

int simple_hash(const Hasher& H, const u64* items, size_t n, u32 mu, std::vector<u64>& T, u32* max_load,
                const uint32_t* values, std::vector<uint32_t>* V) {
  const u32 b = 1u << H.logb;
  std::vector<u64> ixl(n);
  std::vector<u32> ibin(3 * n);
  parallel_ranges(n, [&](size_t lo, size_t hi) {
    for (size_t u = lo; u < hi; ++u) H(items[u], &ixl[u], &ibin[3 * u]);
  });
  // arrivals (bin, x_L) in order: item by item, each distinct bin of the item once
  std::vector<u32> abin, aown;  // bin and item of each arrival
  std::vector<u64> axl;
  abin.reserve(3 * n);
  axl.reserve(3 * n);
  if (V) aown.reserve(3 * n);
  for (size_t u = 0; u < n; ++u) {
    const u64 xl = ixl[u];
    const u32* bs = &ibin[3 * u];
    for (int i = 0; i < 3; ++i) {
      if ((i > 0 && bs[i] == bs[0]) || (i > 1 && bs[i] == bs[1])) continue;
      abin.push_back(bs[i]);
      axl.push_back(xl);
      if (V) aown.push_back((u32)u);
    }
  }
  // stable counting sort by bin keeps the arrival order inside each bin
  std::vector<size_t> off(b + 1, 0);
  for (u32 x : abin) ++off[x + 1];
  for (u32 i = 0; i < b; ++i) off[i + 1] += off[i];
  std::vector<size_t> fill(off.begin(), off.end() - 1);
  std::vector<u64> vals(abin.size());
  std::vector<u32> owners(V ? abin.size() : 0);
  for (size_t e = 0; e < abin.size(); ++e) {
    const size_t at = fill[abin[e]]++;
    vals[at] = axl[e];
    if (V) owners[at] = aown[e];
  }
  // per bin: first arrival of each x_L kept (sorting (x_L, arrival) pairs)
  T.assign((size_t)mu * b, PEPSI_DUMMY);
  if (V) V->assign((size_t)mu * b, 0u);
  std::vector<u32> load(b, 0);
  parallel_ranges(b, [&](size_t blo, size_t bhi) {
    std::vector<std::pair<u64, u32>> tmp;
    std::vector<char> dup;
    for (size_t bin = blo; bin < bhi; ++bin) {
      const size_t s0 = off[bin], len = off[bin + 1] - s0;
      tmp.resize(len);
      dup.assign(len, 0);
      for (size_t r = 0; r < len; ++r) tmp[r] = {vals[s0 + r], (u32)r};
      std::sort(tmp.begin(), tmp.end());
      for (size_t r = 1; r < len; ++r)
        if (tmp[r].first == tmp[r - 1].first) dup[tmp[r].second] = 1;
      u32 layer = 0;
      for (size_t r = 0; r < len; ++r) {
        if (dup[r]) continue;
        if (layer < mu) {
          T[(size_t)layer * b + bin] = vals[s0 + r];
          if (V) (*V)[(size_t)layer * b + bin] = values[owners[s0 + r]];
        }
        ++layer;
      }
      load[bin] = layer;
    }
  });
  const u32 mx = *std::max_element(load.begin(), load.end());
  if (max_load) *max_load = mx;
  return mx > mu ? PEPSI_E_BIN_OVERFLOW : 0;
}

}  // namespace hostmath

namespace hostmath {

// Table 3: the smallest (log2 N, log2 q) for each range of Hamming weights.
bool table3(u32 h, u32* log2n, u32* log2q) {
  static const u32 rows[][4] = {{1, 1, 12, 72},   {2, 2, 13, 144},   {3, 4, 13, 168},  {5, 8, 13, 204},
                                {9, 16, 14, 240}, {17, 32, 14, 276}, {33, 64, 14, 312}};
  for (const auto& r : rows)
    if (h >= r[0] && h <= r[1]) {
      *log2n = r[2];
      *log2q = r[3];
      return true;
    }
  return false;
}

// Eq. 1 without a cap on ell: the smallest ell with C(ell, h) >= 2^lambda_bar
// (C(ell, h) grows with ell, so a binary search over [h, h + 2^lambda_bar]).
u64 code_length_any(u32 lambda_bar, u32 h) {
  if (h == 0 || lambda_bar > 62) return 0;
  const u64 need = 1ull << lambda_bar;
  u64 lo = h, hi = (u64)h + need;
  while (lo < hi) {
    const u64 mid = lo + (hi - lo) / 2;
    if (binom_sat(mid, h) >= need)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

}  // namespace hostmath
