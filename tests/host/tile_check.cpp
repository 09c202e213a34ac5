// tile_check.cpp -- host check of the coalesced tile copies of compiled
// register chains (no GPU).  For every chain of several programs that has a
// tile map (5 or 6 register legs), simulates the copies of warp tiles (lane
// copies tile words lane + 32 i) and checks that every shared-memory slot is written once,
// that the slot each thread reads for its element (tau, e) holds the word at
// base(tau) + hi_off[e], and that no warp instruction (copy or read) has two
// lanes on one bank.  Exit status 0 when all hold.
#include <cstdio>
#include <map>
#include <random>
#include "jit.h"
#include "program.h"
namespace tn {
size_t trace_smem_bytes(const ChainParams &p, size_t elem) { return elem * ((size_t)(p.ngates + 1) * p.tile + 20 * 64); }
size_t chain_smem_bytes(const ChainParams &, size_t) { return 0; }
}
using namespace tn;
static int64_t rc_base(const ChainParams &p, int64_t tau) {
  int64_t base = 0, t = tau;
  for (int sg = p.nseg - 1; sg >= 0; --sg) { base += (t & (p.seg_size[sg] - 1)) << p.seg_ssh[sg]; t >>= p.seg_sh[sg]; }
  return base;
}
static Net square(int L) {
  Net n; n.n = L * L; n.q = 2;
  for (int i = 0; i < L; ++i) for (int j = 0; j < L; ++j) { int s = i * L + j;
    if (j + 1 < L) { n.eu.push_back(s); n.ev.push_back(s + 1); }
    if (i + 1 < L) { n.eu.push_back(s); n.ev.push_back(s + L); } }
  n.m = (int)n.eu.size(); for (int e = 0; e < n.m; ++e) n.J.push_back(1.f);
  for (int i = 0; i < n.n; ++i) n.h.push_back(0.5f);
  n.build_leaves(); return n;
}
int main() {
  std::mt19937_64 rng(9);
  int chains = 0, bad = 0, conflicts = 0;
  for (int L : {16, 20, 24}) for (int ord : {0, 1}) {
    Net net = square(L);
    Tree t; std::string err;
    if (ord == 0) { std::vector<int> seq(net.n); for (int i = 0; i < net.n; ++i) seq[i] = i; tree_from_sweep(net, seq, &t, &err); }
    else { CostModel cm; tree_greedy(net, 5, 4, cm, &t, &err); }
    Plan pl; if (!classify(net, t, &pl, &err)) return 2;
    Program pg; if (!build_program(net, pl, PM_CONFIG, DT_F32, 0, 0, &pg, &err)) return 2;
    for (const ChainParams &p : pg.chains) {
      TileMap tm;
      if (!tile_map(p, &tm)) continue;
      chains++;
      const int RB = p.t, E = 1 << RB;
      const int64_t ntiles = p.outer / 32;
      for (int trial = 0; trial < 8; ++trial) {
        const int64_t t0 = (int64_t)(rng() % (uint64_t)ntiles) * 32;
        std::vector<int64_t> slot(32 * E, -1);
        int Dt[32];
        for (int lane = 0; lane < 32; ++lane) {
          Dt[lane] = 0;
          for (int j = 0; j < 5; ++j) if ((lane >> j) & 1) Dt[lane] ^= tm.cbit[j];
        }
        for (int i = 0; i < E; ++i) {
          int64_t Ci = 0; int Di = 0;
          for (int k = 0; k < RB; ++k) if ((i >> k) & 1) { Ci += int64_t(1) << tm.tpos[5 + k]; Di ^= tm.cbit[5 + k]; }
          bool used[32] = {false};
          for (int lane = 0; lane < 32; ++lane) {
            const int d = Dt[lane] ^ Di;
            if (d < 0 || d >= 32 * E || slot[d] != -1) { bad++; continue; }
            slot[d] = rc_base(p, t0) + lane + Ci;
            if (used[d & 31]) conflicts++;
            used[d & 31] = true;
          }
        }
        for (int e = 0; e < E; ++e) {
          int g = 0;
          for (int b = 0; b < RB; ++b) if ((e >> b) & 1) g ^= tm.gbit[b];
          bool used[32] = {false};
          for (int lane = 0; lane < 32; ++lane) {
            const int d = (e << 5) | (lane ^ g);
            if (slot[d] != rc_base(p, t0 + lane) + p.hi_off[e]) bad++;
            if (used[d & 31]) conflicts++;
            used[d & 31] = true;
          }
        }
      }
    }
  }
  printf("chains %d wrong %d bank_conflicts %d\n", chains, bad, conflicts);
  return (bad || conflicts || chains == 0) ? 1 : 0;
}
