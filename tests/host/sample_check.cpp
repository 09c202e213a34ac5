// Host check of the ground-state sampler (sampler.cpp) with brute-force
// counts: every sample is a ground state, the ground states come out with
// equal frequency, the result does not depend on the batch size, and the
// big-integer helpers are exact.  Prints "ok" lines and exits 0 on success.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <vector>

#include "sampler.h"

using namespace tn;

struct Inst {
  int n;
  std::vector<int> u, v;
  std::vector<float> J, h;
};

static double energy(const Inst &I, const std::vector<float> &h, unsigned x) {
  // x bit i set <-> sigma_i = -1 (state index 1), Eq. 1
  auto s = [&](int i) { return (x >> i & 1) ? -1.0 : 1.0; };
  double E = 0;
  for (size_t e = 0; e < I.u.size(); ++e) E -= I.J[e] * s(I.u[e]) * s(I.v[e]);
  for (int i = 0; i < I.n; ++i) E -= h[i] * s(i);
  return E;
}

static int g_calls = 0;

static CountFn brute(const Inst &I) {
  return [&I](const std::vector<float> &h, int K, std::vector<double> *E, std::vector<Big> *cnt) {
    ++g_calls;
    E->assign(K, 0);
    cnt->assign(K, Big());
    for (int k = 0; k < K; ++k) {
      std::vector<float> hk(h.begin() + (size_t)k * I.n, h.begin() + (size_t)(k + 1) * I.n);
      double best = INFINITY;
      uint64_t c = 0;
      for (unsigned x = 0; x < (1u << I.n); ++x) {
        const double e = energy(I, hk, x);
        if (e < best) { best = e; c = 1; }
        else if (e == best) ++c;
      }
      (*E)[k] = best;
      (*cnt)[k] = Big{c};
    }
    return 0;
  };
}

static int fail(const char *msg) {
  std::printf("FAIL %s\n", msg);
  return 1;
}

static int check_instance(const Inst &I, int S, uint64_t seed, const std::vector<int> &order,
                          const char *name) {
  // the ground states by brute force
  std::map<unsigned, int> gs;
  double Emin = INFINITY;
  for (unsigned x = 0; x < (1u << I.n); ++x) Emin = std::fmin(Emin, energy(I, I.h, x));
  for (unsigned x = 0; x < (1u << I.n); ++x)
    if (energy(I, I.h, x) == Emin) gs[x] = 0;
  std::vector<int8_t> a, b;
  std::string err;
  if (sample_ground_states(I.n, S, order, I.h, seed, 16, brute(I), &a, &err))
    return fail(err.c_str());
  if (sample_ground_states(I.n, S, order, I.h, seed, 3, brute(I), &b, &err))
    return fail(err.c_str());
  if (a != b) return fail("samples depend on the batch size");
  for (int s = 0; s < S; ++s) {
    unsigned x = 0;
    for (int i = 0; i < I.n; ++i) {
      const int8_t v = a[(size_t)s * I.n + i];
      if (v != 1 && v != -1) return fail("sample value not +-1");
      if (v == -1) x |= 1u << i;
    }
    auto it = gs.find(x);
    if (it == gs.end()) return fail("a sample is not a ground state");
    it->second++;
  }
  // Pearson chi-square against the uniform distribution over the ground states
  const double expct = (double)S / gs.size();
  double chi2 = 0;
  int seen = 0;
  for (auto &kv : gs) {
    chi2 += (kv.second - expct) * (kv.second - expct) / expct;
    seen += kv.second > 0;
  }
  const double dof = (double)gs.size() - 1;
  // mean dof, sd sqrt(2 dof): allow 5 sd
  const bool ok = chi2 <= dof + 5 * std::sqrt(2 * dof) + 1 && seen == (int)gs.size();
  std::printf("%s ground_states %zu samples %d chi2 %.2f dof %.0f %s\n", name, gs.size(), S, chi2,
              dof, ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}

int main() {
  int bad = 0;
  // big-integer helpers
  {
    Big a{~0ull, 1}, b{1};
    Big c = big_add(a, b);
    if (!(c.size() == 2 && c[0] == 0 && c[1] == 2)) bad += fail("big_add carry");
    if (!big_less(b, a) || big_less(a, b) || big_less(a, a)) bad += fail("big_less");
    if (!big_less(Big{5}, Big{5, 0, 1})) bad += fail("big_less length");
    if (big_less(Big{5, 0}, Big{5})) bad += fail("big_less leading zero");
    Big bound{7, 1};   // 2^64 + 7
    for (uint64_t t = 0; t < 2000; ++t) {
      Big r = uniform_below(bound, 3, 1, t);
      if (!big_less(r, bound)) { bad += fail("uniform_below out of range"); break; }
    }
    std::vector<int> hist(6, 0);
    for (uint64_t t = 0; t < 60000; ++t) {
      Big r = uniform_below(Big{6}, 9, t, 0);
      hist[r.empty() ? 0 : r[0]]++;
    }
    for (int k = 0; k < 6; ++k)
      if (std::abs(hist[k] - 10000) > 500) { bad += fail("uniform_below not uniform"); break; }
    std::printf("helpers %s\n", bad ? "FAIL" : "ok");
  }
  // frustrated ring of 7 spins, one antiferromagnetic bond: 14 ground states
  {
    Inst I{7, {}, {}, {}, std::vector<float>(7, 0.f)};
    for (int i = 0; i < 7; ++i) {
      I.u.push_back(i);
      I.v.push_back((i + 1) % 7);
      I.J.push_back(i == 0 ? -1.f : 1.f);
    }
    std::vector<int> order{3, 0, 6, 1, 5, 2, 4};
    bad += check_instance(I, 1400, 11, order, "ring7");
  }
  // +-J 3 x 3 lattice with an integer field; the first coupling draw with at
  // least 4 ground states
  {
    for (uint64_t seed = 1;; ++seed) {
      Inst I{9, {}, {}, {}, std::vector<float>(9, 0.f)};
      for (int y = 0; y < 3; ++y)
        for (int x = 0; x < 3; ++x) {
          const int i = 3 * y + x;
          if (x + 1 < 3) { I.u.push_back(i); I.v.push_back(i + 1); }
          if (y + 1 < 3) { I.u.push_back(i); I.v.push_back(i + 3); }
        }
      uint64_t r = seed;
      for (size_t e = 0; e < I.u.size(); ++e) {
        r = mix64(r);
        I.J.push_back((r & 1) ? 1.f : -1.f);
      }
      I.h[4] = 1.f;
      double Emin = INFINITY;
      int c = 0;
      for (unsigned x = 0; x < 512; ++x) {
        const double e = energy(I, I.h, x);
        if (e < Emin) { Emin = e; c = 1; } else if (e == Emin) ++c;
      }
      if (c < 4) continue;
      std::vector<int> order{8, 7, 6, 5, 4, 3, 2, 1, 0};
      bad += check_instance(I, 1200, 5, order, "pm3x3");
      break;
    }
  }
  // a single ground state (ferromagnetic chain with a field)
  {
    Inst I{5, {0, 1, 2, 3}, {1, 2, 3, 4}, {1.f, 1.f, 1.f, 1.f}, {0.f, 0.f, 1.f, 0.f, 0.f}};
    std::vector<int> order{0, 1, 2, 3, 4};
    bad += check_instance(I, 50, 1, order, "ferro5");
  }
  std::printf("calls %d bad %d\n", g_calls, bad);
  return bad ? 1 : 0;
}
