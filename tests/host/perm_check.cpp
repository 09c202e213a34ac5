// perm_check.cpp -- host check of the tiled q = 2 transpose (perm_bits.h,
// k_permute2).  For random permutations of the legs of tensors with 1..26
// legs (each leg of dimension 2, runs of legs merged as the lowering merges
// them), simulates the kernel's index arithmetic: every output element is
// written exactly once, from the input element the permutation defines
// (out[o] = in[sum_j i_j sin_j]); every tile slot is filled before it is read;
// and in both phases the 32 lanes of a warp touch 32 consecutive global
// elements and 32 distinct shared-memory banks.  Exit status 0 when all hold.
#include <cstdio>
#include <random>
#include <vector>
#include <algorithm>

#include "perm_bits.h"

using namespace tn;

static int swz(const PermBits &pb, int L) {
  for (int i = 0; i < pb.nsw; ++i) L ^= ((L >> (5 + pb.sw_row[i])) & 1) << pb.sw_bank[i];
  return L;
}

int main() {
  std::mt19937_64 rng(11);
  int cases = 0, bad = 0, conflicts = 0, uncoalesced = 0;
  for (int trial = 0; trial < 400; ++trial) {
    const int n = 1 + (int)(rng() % 26);
    // input legs 0..n-1 (leg l has stride 2^l); output order = a permutation
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::shuffle(perm.begin(), perm.end(), rng);
    if (trial % 4 == 0) std::sort(perm.begin(), perm.end());   // identity-like runs too
    // output legs listed slowest first: to[j] is an input leg; merge runs as
    // the lowering does (adjacent in the input too)
    std::vector<int64_t> md, ms;
    for (int j = 0; j < n; ++j) {
      const int64_t d = 2, s = int64_t(1) << perm[j];
      if (!md.empty() && ms.back() == s * d) { md.back() *= d; ms.back() = s; }
      else { md.push_back(d); ms.push_back(s); }
    }
    PermParams p{};
    p.r = (int)md.size();
    p.total = int64_t(1) << n;
    for (int j = 0; j < p.r; ++j) { p.dims[j] = md[j]; p.sin[j] = ms[j]; }
    PermBits pb;
    if (!perm_bits(p, &pb)) { bad++; continue; }
    cases++;
    // reference: input offset of output element o
    std::vector<int64_t> ref(p.total);
    for (int64_t o = 0; o < p.total; ++o) {
      int64_t r = o, off = 0;
      for (int j = p.r - 1; j >= 0; --j) { off += (r % p.dims[j]) * p.sin[j]; r /= p.dims[j]; }
      ref[o] = off;
    }
    std::vector<int> written(p.total, 0);
    const int nt = 1 << pb.nT;
    const int64_t tiles_to_check = std::min<int64_t>(pb.tiles, 64);
    for (int64_t tt = 0; tt < pb.tiles; ++tt) {
      const int64_t tau = tt < tiles_to_check ? tt : (int64_t)(rng() % (uint64_t)pb.tiles);
      int64_t bin = 0, bout = 0;
      for (int g = 0; g < pb.nseg; ++g) {
        const int64_t v = (tau >> pb.seg_t[g]) & ((int64_t(1) << pb.seg_len[g]) - 1);
        bin += v << pb.seg_in[g];
        bout += v << pb.seg_out[g];
      }
      std::vector<int64_t> slot(nt, -1);
      for (int w = 0; w < (nt + 31) / 32; ++w) {
        bool bank[32] = {false};
        int64_t first = -1;
        for (int lane = 0; lane < 32 && w * 32 + lane < nt; ++lane) {
          const int j = w * 32 + lane;
          int L = 0;
          int64_t off = 0;
          for (int t = 0; t < pb.nT; ++t)
            if ((j >> t) & 1) { L |= 1 << pb.rd_local[t]; off += int64_t(1) << pb.rd_in[t]; }
          const int s = swz(pb, L);
          if (s < 0 || s >= nt || slot[s] != -1) { bad++; continue; }
          slot[s] = bin + off;
          if (bank[s & 31]) conflicts++;
          bank[s & 31] = true;
          if (lane == 0) first = bin + off;
          else if (nt >= 32 && bin + off != first + lane) uncoalesced++;
        }
      }
      for (int w = 0; w < (nt + 31) / 32; ++w) {
        bool bank[32] = {false};
        int64_t first = -1;
        for (int lane = 0; lane < 32 && w * 32 + lane < nt; ++lane) {
          const int j = w * 32 + lane;
          int64_t off = 0;
          for (int t = 0; t < pb.nT; ++t)
            if ((j >> t) & 1) off += int64_t(1) << pb.wr_out[t];
          const int64_t o = bout + off;
          const int s = swz(pb, j);
          if (o < 0 || o >= p.total || s < 0 || s >= nt || slot[s] != ref[o]) { bad++; continue; }
          if (tt < tiles_to_check || pb.tiles <= 64) written[o]++;
          if (bank[s & 31]) conflicts++;
          bank[s & 31] = true;
          if (lane == 0) first = o;
          else if (nt >= 32 && o != first + lane) uncoalesced++;
        }
      }
      if (tt >= tiles_to_check) break;   // large tensors: 64 tiles in order + one random
    }
    if (pb.tiles <= 64)
      for (int64_t o = 0; o < p.total; ++o)
        if (written[o] != 1) { bad++; break; }
  }
  printf("cases %d wrong %d bank_conflicts %d uncoalesced %d\n", cases, bad, conflicts, uncoalesced);
  return (bad || conflicts || uncoalesced || cases == 0) ? 1 : 0;
}
