// tile_check.cpp -- host check of the coalesced tile copies of compiled
// register chains (no GPU).  For every chain of several programs and both of
// its layouts (input: hi_in / ssh_in, output: hi_out / ssh_out), simulates a
// warp tile: lane copies tile words lane + 32 i, i < 2^nreg, between memory
// (tile base + lane + off_i) and shared-memory slot D_lane ^ D_i.  Checks that
// every slot is used once, that the slot the thread of lane uses for register
// state e (tile_slot) holds the element at base(tau) + hi[e] of that layout,
// and that no warp instruction (copy, or the owners' accesses for one e) has
// two lanes on one bank.  The vector copies (tile_vec: w words per lane when
// memory positions below log2 w map to slot bits below log2 w) must move the
// same words to the same slots, w-aligned in memory and in shared memory, with
// the lanes of each wavefront (32 / w of them) on distinct bank groups; the
// owners move the 2^a states that differ in the low register legs (memory
// positions 0..a-1) as one vector, conflict-free in the same sense.  Programs include chains that start from a
// rank-raising step (the new leg is not a leg of the input) and chains that
// end with a contraction (the contracted leg is not a leg of the output).
// Exit status 0 when all hold.
#include <cstdio>
#include <algorithm>
#include <map>
#include <random>
#include "jit.h"
#include "program.h"
namespace tn {
size_t trace_smem_bytes(const ChainParams &p, size_t elem) { return elem * ((size_t)(p.ngates + 1) * p.tile + 20 * 64); }
size_t chain_smem_bytes(const ChainParams &, size_t) { return 0; }
}
using namespace tn;
static int64_t base_of(const ChainParams &p, int64_t tau, const int32_t *ssh) {
  int64_t base = 0, t = tau;
  for (int sg = p.nseg - 1; sg >= 0; --sg) { base += (t & (p.seg_size[sg] - 1)) << ssh[sg]; t >>= p.seg_sh[sg]; }
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
  int chains = 0, sides = 0, partial = 0, bad = 0, conflicts = 0, vbad = 0, vsides = 0, lowsides = 0;
  for (int L : {16, 20, 24}) for (int ord : {0, 1, 2, 3}) for (int mode : {0, 1}) {
    Net net = square(L);
    Tree t; std::string err;
    if (ord == 0) { std::vector<int> seq(net.n); for (int i = 0; i < net.n; ++i) seq[i] = i; tree_from_sweep(net, seq, &t, &err); }
    else { CostModel cm; tree_greedy(net, 5 + ord, 4, cm, &t, &err); }
    Plan pl; if (!classify(net, t, &pl, &err)) return 2;
    Program pg; if (!build_program(net, pl, (ProgMode)mode, DT_F32, 0, 0, &pg, &err)) return 2;
    for (const ChainParams &p : pg.chains) {
      if (p.mode != 1 || p.P != 0) continue;
      chains++;
      for (int side = 0; side < 2; ++side) {
        const int64_t *hi = side == 0 ? p.hi_in : p.hi_out;
        const int32_t *ssh = side == 0 ? p.ssh_in : p.ssh_out;
        TileMap tm;
        if (!tile_map(p, hi, &tm)) { bad++; continue; }
        sides++;
        partial += tm.nreg < p.t;
        const int E = 1 << p.t, N = 1 << tm.nreg;
        const int64_t ntiles = p.outer / 32;
        for (int trial = 0; trial < 6; ++trial) {
          const int64_t t0 = (int64_t)(rng() % (uint64_t)ntiles) * 32;
          std::vector<int64_t> slot(32 * N, -1);
          for (int i = 0; i < N; ++i) {
            int Di; int64_t off;
            tile_word(tm, i, &Di, &off);
            bool used[32] = {false};
            for (int lane = 0; lane < 32; ++lane) {
              int Dl = 0;
              for (int j = 0; j < 5; ++j) if ((lane >> j) & 1) Dl ^= tm.cbit[j];
              const int d = Dl ^ Di;
              if (d < 0 || d >= 32 * N || slot[d] != -1) { bad++; continue; }
              slot[d] = base_of(p, t0, ssh) + lane + off;
              if (used[d & 31]) conflicts++;
              used[d & 31] = true;
            }
          }
          // vector copies (tile_vec): the same words and slots, w at a time
          const int w = tile_vec(tm);
          std::vector<int> vseen(32 * N, 0);
          bool vused[32] = {false};
          for (int i = 0; i < N; i += w) {
            int Di; int64_t offi;
            tile_word(tm, i, &Di, &offi);
            for (int lane = 0; lane < 32; ++lane) {
              int Dv; int64_t ov;
              tile_vec_lane(tm, w, lane, &Dv, &ov);
              const int s0 = Dv ^ Di;
              if (s0 % w || (ov + offi) % w) vbad++;
              // one wavefront per group of 32 / w lanes: distinct bank groups
              if (lane % (32 / w) == 0) std::fill(vused, vused + 32, false);
              if (vused[(s0 / w) % (32 / w)]) conflicts++;
              vused[(s0 / w) % (32 / w)] = true;
              for (int j = 0; j < w; ++j) {
                const int line = i + lane / (32 / w), word = (lane % (32 / w)) * w + j;
                int Dl = 0;
                for (int b = 0; b < 5; ++b) if ((word >> b) & 1) Dl ^= tm.cbit[b];
                int Dline; int64_t offline;
                tile_word(tm, line, &Dline, &offline);
                if (s0 + j != (Dl ^ Dline) || ov + offi + j != word + offline) vbad++;
                if (s0 + j >= 0 && s0 + j < 32 * N) vseen[s0 + j]++;
              }
            }
          }
          for (int v : vseen) if (v != 1) vbad++;
          if (trial == 0) vsides += w > 1;
          // owners' accesses: the 2^a states that differ in the low legs form
          // one aligned vector of the thread; the lanes of each group of
          // 32 / 2^a (one wavefront) hit distinct bank groups
          const int A = 1 << tm.a;
          for (int e = 0; e < E; ++e) {
            bool used[32] = {false};
            for (int lane = 0; lane < 32; ++lane) {
              const int d = tile_slot(tm, lane, e);
              if (d < 0 || d >= 32 * N || slot[d] != base_of(p, t0 + lane, ssh) + hi[e]) bad++;
              if ((d & (A - 1)) != (tile_slot(tm, 0, e) & (A - 1))) bad++;
              if (lane % (32 / A) == 0) std::fill(used, used + 32, false);
              const int bg = (d / A) % (32 / A);
              if (used[bg]) conflicts++;
              used[bg] = true;
            }
          }
          lowsides += trial == 0 && tm.a > 0;
        }
      }
    }
  }
  // the generated kernels of chains with low register legs compile (NVRTC,
  // FP32 and INT32 forms; no device needed)
  int compiled = 0, compile_fail = 0;
  {
    Net net = square(24);
    Tree t; std::string err; CostModel cm;
    tree_greedy(net, 7, 4, cm, &t, &err);
    Plan pl; if (!classify(net, t, &pl, &err)) return 2;
    for (Dtype dt : {DT_F32, DT_I32}) {
      Program pg; if (!build_program(net, pl, PM_ENERGY, dt, 0, 0, &pg, &err)) return 2;
      int n = 0;
      for (const ChainParams &p : pg.chains) {
        TileMap a, b;
        if (p.mode != 1 || p.P != 0 || !tile_map(p, p.hi_in, &a) || !tile_map(p, p.hi_out, &b)) continue;
        if (a.a == 0 && b.a == 0) continue;
        if (n++ >= 3) break;
        const std::string name = "tn_chain_check" + std::to_string(compiled + compile_fail);
        const std::string src = jit_chain_source(p, dt, name);
        std::string cubin, cerr;
        if (!src.empty() && jit_compile_source(src, name, &cubin, &cerr)) compiled++;
        else { compile_fail++; fprintf(stderr, "%s\n", cerr.c_str()); }
      }
    }
  }
  printf("generated kernels with low register legs: compiled %d failed %d\n", compiled, compile_fail);
  if (compiled == 0 || compile_fail) return 1;
  printf("vector copies: layouts %d wrong %d; layouts with low register legs %d\n", vsides, vbad,
         lowsides);
  printf("chains %d layouts %d (without a register leg: %d) wrong %d bank_conflicts %d\n", chains,
         sides, partial, bad, conflicts);
  return (bad || conflicts || vbad || chains == 0 || vsides == 0 || lowsides == 0) ? 1 : 0;
}
