// sampler.cpp -- ground states drawn by conditional counts (see sampler.h).
#include "sampler.h"

#include <algorithm>

namespace tn {

uint64_t mix64(uint64_t x) {
  // SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014)
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

static void trim(Big *a) {
  while (!a->empty() && a->back() == 0) a->pop_back();
}

bool big_less(const Big &a0, const Big &b0) {
  Big a = a0, b = b0;
  trim(&a);
  trim(&b);
  if (a.size() != b.size()) return a.size() < b.size();
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i];
  return false;
}

Big big_add(const Big &a, const Big &b) {
  Big r(std::max(a.size(), b.size()) + 1, 0);
  uint64_t carry = 0;
  for (size_t i = 0; i + 1 < r.size(); ++i) {
    const uint64_t x = i < a.size() ? a[i] : 0, y = i < b.size() ? b[i] : 0;
    const uint64_t s = x + y;
    const uint64_t c1 = s < x ? 1 : 0;
    r[i] = s + carry;
    const uint64_t c2 = r[i] < s ? 1 : 0;
    carry = c1 + c2;
  }
  r.back() = carry;
  trim(&r);
  return r;
}

// Uniform integer in [0, bound) by rejection: draw as many random bits as
// bound has and retry while the draw is not below it (fewer than two draws
// expected).  bound must be nonzero.
Big uniform_below(const Big &bound0, uint64_t seed, uint64_t s, uint64_t step) {
  Big bound = bound0;
  trim(&bound);
  const size_t L = bound.size();
  const uint64_t top = bound.back();
  int bits = 0;
  while (bits < 64 && (top >> bits) != 0) ++bits;
  const uint64_t mask = bits == 64 ? ~0ull : ((1ull << bits) - 1);
  const uint64_t key = mix64(mix64(mix64(seed) ^ s) ^ step);
  for (uint64_t attempt = 0;; ++attempt) {
    Big r(L);
    for (size_t i = 0; i < L; ++i) r[i] = mix64(key ^ mix64((attempt << 16) | i));
    r[L - 1] &= mask;
    if (big_less(r, bound)) {
      trim(&r);
      return r;
    }
  }
}

int sample_ground_states(int n, int S, const std::vector<int> &order, const std::vector<float> &h0,
                         uint64_t seed, int chunk, const CountFn &count,
                         std::vector<int8_t> *sigma, std::string *err) {
  sigma->assign((size_t)S * n, 0);
  if (S == 0) return 0;
  if ((int)order.size() != n || (int)h0.size() != n || chunk < 1) {
    *err = "sampler: bad order, fields or chunk";
    return -1;
  }
  // the unpinned instance: E_min
  std::vector<double> E;
  std::vector<Big> C;
  int rc = count(h0, 1, &E, &C);
  if (rc) return rc;
  const double Emin = E[0];
  if (!big_less(Big{}, C[0])) {
    *err = "sampler: the instance has no ground state";
    return -1;
  }
  for (int s0 = 0; s0 < S; s0 += chunk) {
    const int cs = std::min(chunk, S - s0);
    std::vector<float> pin((size_t)cs * n, 0.0f);   // pin field of each sample
    std::vector<float> h((size_t)2 * cs * n);
    for (int t = 0; t < n; ++t) {
      const int i = order[t];
      for (int s = 0; s < cs; ++s)
        for (int c = 0; c < 2; ++c) {
          float *hk = h.data() + (size_t)(2 * s + c) * n;
          for (int j = 0; j < n; ++j) hk[j] = h0[j] + pin[(size_t)s * n + j];
          hk[i] = h0[i] + (c == 0 ? 1.0f : -1.0f);
        }
      rc = count(h, 2 * cs, &E, &C);
      if (rc) return rc;
      const double target = Emin - (double)(t + 1);
      for (int s = 0; s < cs; ++s) {
        const Big wp = E[2 * s] == target ? C[2 * s] : Big{};
        const Big wm = E[2 * s + 1] == target ? C[2 * s + 1] : Big{};
        const Big tot = big_add(wp, wm);
        if (tot.empty()) {
          *err = "sampler: no ground state extends the fixed spins (inconsistent counts)";
          return -1;
        }
        const Big r = uniform_below(tot, seed, (uint64_t)(s0 + s), (uint64_t)t);
        const int8_t v = big_less(r, wp) ? 1 : -1;
        pin[(size_t)s * n + i] = (float)v;
        (*sigma)[(size_t)(s0 + s) * n + i] = v;
      }
    }
  }
  return 0;
}

}  // namespace tn
