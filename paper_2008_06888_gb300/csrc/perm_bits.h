// perm_bits.h -- index-bit map of a q = 2 tensor permutation for the tiled
// transpose kernel (k_permute2).  Host code; shared with the host-side check
// tests/host/perm_check.cpp.
#pragma once
#include <stdint.h>

#include "tn_internal.h"

namespace tn {

// ---- q = 2: a permutation of the legs is a permutation of the index bits.
// Tiled transpose through shared memory: a tile spans the output's 5 lowest
// bits (the write lanes), the output bits holding the input's 5 lowest bits
// (the read lanes) and more low output bits up to 2^10 elements; the other
// output bits number the tiles.  Both the reads and the writes of a warp move
// 32 consecutive elements, and the shared-memory index is XOR-swizzled so
// neither phase has two lanes on one bank.
struct PermBits {
  int nT;                      // tile bits
  int rd_local[10], rd_in[10]; // read bit t -> tile-local bit, input bit
  int wr_out[10];              // tile-local bit t -> output bit
  int nsw, sw_row[5], sw_bank[5];  // local bit 5 + sw_row[i] flips bank bit sw_bank[i]
  int nseg;                    // outer bits: runs consecutive in output and input
  int seg_t[TN_MAX_RANK], seg_len[TN_MAX_RANK], seg_in[TN_MAX_RANK], seg_out[TN_MAX_RANK];
  int64_t tiles;
};

inline bool perm_bits(const PermParams &p, PermBits *pb) {
  int ip[64], nbits = 0;
  for (int j = p.r - 1; j >= 0; --j) {
    int a = 0, s = 0;
    while ((int64_t(1) << a) < p.dims[j]) ++a;
    while ((int64_t(1) << s) < p.sin[j]) ++s;
    if ((int64_t(1) << a) != p.dims[j] || (int64_t(1) << s) != p.sin[j]) return false;
    for (int t = 0; t < a; ++t) {
      if (nbits >= 62) return false;
      ip[nbits++] = s + t;
    }
  }
  if ((int64_t(1) << nbits) != p.total) return false;
  int inv[64];
  for (int k = 0; k < nbits; ++k) {
    if (ip[k] < 0 || ip[k] >= nbits) return false;
    inv[ip[k]] = k;
  }
  bool inT[64] = {false};
  const int m = nbits < 5 ? nbits : 5;
  int nT = 0;
  for (int k = 0; k < m; ++k) inT[k] = true;
  for (int u = 0; u < m; ++u) inT[inv[u]] = true;
  for (int k = 0; k < nbits; ++k) nT += inT[k];
  for (int k = 0; k < nbits && nT < 10; ++k)
    if (!inT[k]) { inT[k] = true; ++nT; }
  *pb = PermBits{};
  pb->nT = nT;
  int rank[64], t = 0;
  for (int k = 0; k < nbits; ++k)
    if (inT[k]) { rank[k] = t; pb->wr_out[t++] = k; }
  bool used[64] = {false};
  t = 0;
  for (int u = 0; u < m; ++u) {
    pb->rd_local[t] = rank[inv[u]];
    pb->rd_in[t++] = u;
    used[inv[u]] = true;
  }
  for (int k = 0; k < nbits; ++k)
    if (inT[k] && !used[k]) {
      pb->rd_local[t] = rank[k];
      pb->rd_in[t++] = ip[k];
    }
  // swizzle: the read lanes' local bits at 5 and above flip the bank bits the
  // read lanes leave fixed
  bool lo[5] = {false, false, false, false, false};
  int hi[5], nhi = 0;
  for (int u = 0; u < m; ++u) {
    if (pb->rd_local[u] < 5) lo[pb->rd_local[u]] = true;
    else hi[nhi++] = pb->rd_local[u] - 5;
  }
  for (int b = 0, i = 0; b < 5 && i < nhi; ++b)
    if (!lo[b]) { pb->sw_row[i] = hi[i]; pb->sw_bank[i] = b; ++i; pb->nsw = i; }
  // outer bits, ascending in the output: runs that are consecutive in both
  int tb = 0;
  for (int k = 0; k < nbits; ++k) {
    if (inT[k]) continue;
    if (pb->nseg > 0) {
      const int g = pb->nseg - 1;
      if (pb->seg_out[g] + pb->seg_len[g] == k && pb->seg_in[g] + pb->seg_len[g] == ip[k]) {
        pb->seg_len[g]++;
        ++tb;
        continue;
      }
    }
    if (pb->nseg == TN_MAX_RANK) return false;
    const int g = pb->nseg++;
    pb->seg_t[g] = tb++;
    pb->seg_len[g] = 1;
    pb->seg_in[g] = ip[k];
    pb->seg_out[g] = k;
  }
  pb->tiles = int64_t(1) << (nbits - nT);
  return true;
}

}  // namespace tn
