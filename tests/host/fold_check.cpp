// fold_check.cpp -- host check of the register-chain fold (no GPU).
//
// Builds the energy and traceback programs of several lattices and chimera
// graphs, then evaluates every register chain twice on sampled outer
// indices: through its original gate list (replace gates: max over the
// eliminated digit of value + operand; diagonal gates: value + operand; a
// final contraction: max over the contracted digit; a chain that starts
// from a rank-raising step reads both states of the new leg from one input
// element) and through its folded table gates.  Operands and inputs are small integers
// drawn from a hash, so both evaluations are exact and must agree exactly.
// Exit status 0 when every chain agrees.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <algorithm>
#include "program.h"
namespace tn {
size_t trace_smem_bytes(const ChainParams &p, size_t elem) { return elem * ((size_t)(p.ngates + 1) * p.tile + 20 * 64); }
size_t chain_smem_bytes(const ChainParams &, size_t) { return 0; }
}
using namespace tn;
static double X(int64_t i) { uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull; h ^= h >> 29; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 32; return (double)(int)(h % 9) - 4.0; }
static int64_t rc_base(const ChainParams &p, int64_t tau, const int32_t *ssh = nullptr) {
  int64_t base = 0, t = tau;
  for (int sg = p.nseg - 1; sg >= 0; --sg) { base += (t & (p.seg_size[sg] - 1)) << (ssh ? ssh[sg] : p.seg_ssh[sg]); t >>= p.seg_sh[sg]; }
  return base;
}
static int check_chain(const ChainParams &p, std::mt19937_64 &rng, int *ntg_out) {
  int bad = 0;
  std::vector<double> T(p.ttotal + 8);
  for (int k = 0; k < p.ntg; ++k) {
    const TGate &t = p.tg[k];
    for (int i = 0; i < (8 << t.nf); ++i) {
      double acc = 0;
      for (int c = 0; c < t.ncomp; ++c) {
        const ChainGate &g = p.g[t.cg[c]];
        const int64_t st[4] = {g.sBk, g.sBn, g.sBb[0], g.sBb[1]};
        int64_t o = 0;
        for (int l = 0; l < 4; ++l) if (t.cbit[c][l] >= 0) o += (int64_t)((i >> t.cbit[c][l]) & 1) * st[l];
        acc += X(g.offB + o);
      }
      T[t.toff + i] = acc;
    }
  }
  for (int trial = 0; trial < 64; ++trial) {
    int64_t tau = (int64_t)(rng() % (uint64_t)p.outer);
    int64_t base = rc_base(p, tau), base_in = rc_base(p, tau, p.ssh_in);
    const int E = p.tile;   // 2^t register states
    double v[64], w[64];
    // input layout: a chain starting with a rank-raising step reads both states
    // of the new leg from one input element
    for (int e = 0; e < E; ++e) v[e] = w[e] = X(1000000007ll + base_in + p.hi_in[e]);
    int cj = -1;   // register bit of a final contraction
    for (int gi = 0; gi < p.ngates; ++gi) {
      const ChainGate &g = p.g[gi];
      auto dig = [&](int k, int e) { return g.lsb[k] >= 0 ? (e >> g.lsb[k]) & 1 : (int)((base >> g.lsbh[k]) & 1); };
      if (g.kind == 2) {   // contraction: state e (bit ls clear) keeps the max over the bit
        cj = g.ls;
        for (int e = 0; e < E; ++e) {
          if (e & (1 << g.ls)) continue;
          int64_t bo = 0;
          for (int l = 0; l < g.nb; ++l) bo += dig(l, e) * g.sBb[l];
          v[e] = std::max(v[e] + X(g.offB + bo), v[e | (1 << g.ls)] + X(g.offB + bo + g.sBk));
        }
      } else if (g.kind != 0) {
        for (int e = 0; e < E; ++e) { int x0 = dig(0, e), x1 = g.nb > 1 ? dig(1, e) : 0; v[e] += X(g.offB + x0 * g.sBb[0] + x1 * (g.nb > 1 ? g.sBb[1] : 0)); }
      } else {
        for (int e = 0; e < E; ++e) {
          if (e & (1 << g.ls)) continue;
          int e1 = e | (1 << g.ls);
          int ww = g.nb > 0 ? dig(0, e) : 0;
          int64_t bo = ww * (g.nb > 0 ? g.sBb[0] : 0);
          double a = v[e], b = v[e1];
          v[e] = std::max(a + X(g.offB + bo), b + X(g.offB + bo + g.sBk));
          v[e1] = std::max(a + X(g.offB + bo + g.sBn), b + X(g.offB + bo + g.sBk + g.sBn));
        }
      }
    }
    for (int k = 0; k < p.ntg; ++k) {
      const TGate &t = p.tg[k];
      int f = 0;
      for (int i = 0; i < t.nf; ++i) f |= (int)((tau >> t.fsh[i]) & 1) << i;
      const double *tab = &T[t.toff + f * 8];
      if (t.kind == 2) {
        for (int e = 0; e < E; ++e) {
          if (e & (1 << t.J)) continue;
          int kk = t.K >= 0 ? (e >> t.K) & 1 : 0;
          w[e] = std::max(w[e] + tab[kk * 4], w[e | (1 << t.J)] + tab[kk * 4 + 1]);
        }
      } else if (t.kind != 0) {
        for (int e = 0; e < E; ++e) { int x0 = t.J >= 0 ? (e >> t.J) & 1 : 0, x1 = t.K >= 0 ? (e >> t.K) & 1 : 0; w[e] += tab[x0 | x1 << 1]; }
      } else {
        for (int e = 0; e < E; ++e) {
          if (e & (1 << t.J)) continue;
          int e1 = e | (1 << t.J); int kk = t.K >= 0 ? (e >> t.K) & 1 : 0;
          double a = w[e], b = w[e1];
          w[e] = std::max(a + tab[kk * 4], b + tab[kk * 4 + 1]);
          w[e1] = std::max(a + tab[kk * 4 + 2], b + tab[kk * 4 + 3]);
        }
      }
    }
    for (int e = 0; e < E; ++e)
      if ((cj < 0 || !(e & (1 << cj))) && v[e] != w[e]) bad++;
  }
  *ntg_out = p.ntg;
  return bad;
}
static Net square(int L, bool field, uint64_t seed) {
  Net n; n.n = L * L; n.q = 2;
  std::mt19937_64 r(seed);
  for (int i = 0; i < L; ++i) for (int j = 0; j < L; ++j) {
    int s = i * L + j;
    if (j + 1 < L) { n.eu.push_back(s); n.ev.push_back(s + 1); }
    if (i + 1 < L) { n.eu.push_back(s); n.ev.push_back(s + L); }
  }
  n.m = (int)n.eu.size();
  for (int e = 0; e < n.m; ++e) n.J.push_back((float)((int)(r() % 3) - 1));
  if (field) for (int i = 0; i < n.n; ++i) n.h.push_back(0.5f);
  n.build_leaves();
  return n;
}
static Net chimera(int L, uint64_t seed) {
  Net n; n.q = 2; n.n = 8 * L * L;
  for (int i = 0; i < L; ++i) for (int j = 0; j < L; ++j) {
    int b = 8 * (i * L + j);
    for (int a = 0; a < 4; ++a) for (int c = 0; c < 4; ++c) { n.eu.push_back(b + a); n.ev.push_back(b + 4 + c); }
    if (i + 1 < L) for (int a = 0; a < 4; ++a) { n.eu.push_back(b + a); n.ev.push_back(8 * ((i + 1) * L + j) + a); }
    if (j + 1 < L) for (int a = 0; a < 4; ++a) { n.eu.push_back(b + 4 + a); n.ev.push_back(8 * (i * L + j + 1) + 4 + a); }
  }
  n.m = (int)n.eu.size();
  for (int e = 0; e < n.m; ++e) n.J.push_back(1.f);
  n.build_leaves();
  return n;
}
int main() {
  std::mt19937_64 rng(5);
  int total_bad = 0, nchains = 0, norig = 0, nfold = 0, ncontract = 0, ngrow = 0;
  struct Case { const char *name; Net net; int order; };
  std::vector<Case> cases;
  for (int L : {14, 20, 24}) { cases.push_back({"sq", square(L, true, L), 0}); cases.push_back({"sqg", square(L, false, L + 1), 1}); cases.push_back({"sqg-f", square(L, true, L + 2), 1}); }
  cases.push_back({"chim", chimera(4, 3), 1});
  for (auto &c : cases) {
    Tree t; std::string err;
    if (c.order == 0) {
      std::vector<int> seq(c.net.n); for (int i = 0; i < c.net.n; ++i) seq[i] = i;
      if (!tree_from_sweep(c.net, seq, &t, &err)) { printf("sweep fail %s\n", err.c_str()); return 1; }
    } else {
      CostModel cm;
      if (!tree_greedy(c.net, 7, 8, cm, &t, &err)) { printf("greedy fail %s\n", err.c_str()); return 1; }
    }
    Plan pl;
    if (!classify(c.net, t, &pl, &err)) { printf("classify fail %s\n", err.c_str()); return 1; }
    for (int mode : {0, 1}) {
      Program pg;
      if (!build_program(c.net, pl, (ProgMode)mode, DT_F32, 0, mode == 1 ? (int64_t)1 << 28 : 0, &pg, &err)) { printf("build fail %s\n", err.c_str()); return 1; }
      auto run = [&](const ChainParams &p) {
        if (p.mode != 1) return;
        int ntg = 0;
        int bad = check_chain(p, rng, &ntg);
        for (int i = 0; i < p.ngates; ++i) ncontract += p.g[i].kind == 2;
        for (int e = 1; e < p.tile; ++e) ngrow += p.hi_in[e] == 0;
        total_bad += bad; nchains++; norig += p.ngates; nfold += ntg;
        if (bad) printf("MISMATCH %s n=%d chain ngates=%d ntg=%d bad=%d\n", c.name, c.net.n, p.ngates, ntg, bad);
      };
      for (auto &p : pg.chains) run(p);
      for (auto &ct : pg.chain_traces) run(ct.p);
    }
  }
  printf("rank-changing: %d contractions, %d grown legs\n", ncontract, ngrow);
  printf("chains %d orig gates %d table gates %d mismatches %d\n", nchains, norig, nfold, total_bad);
  return total_bad != 0;
}
