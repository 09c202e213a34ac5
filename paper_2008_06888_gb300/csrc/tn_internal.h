// tn_internal.h -- structures shared by the host planner/executor and the
// CUDA kernels of libtn.so.  Not part of the public ABI (include/tn.h).
#pragma once
#include <stdint.h>

#define TN_MAX_SEG 10        // outer-index segments of a gate contraction
#define TN_GATE_MAX_K 64     // contracted states of a gate contraction
#define TN_GATE_MAX_N 16     // new (N) states of a gate contraction
#define TN_MAX_RANK 40       // legs of one tensor
#define TN_MAX_PRIMES 9      // residue planes of a counting tensor (incl. witness)
#define TN_MAX_TRACE_LEGS 40

// Element offsets are int64; every tensor has q^rank elements.

// C[o, n] = max_k A[o, k] + B[o, k, n] over the outer index o (batch and M
// legs of C), the contracted states k (K legs) and the new states n (N legs).
// The outer index is split into segments (slowest first); each segment has
// one stride per operand.  Offsets of k and n are tabulated.
struct GateParams {
  int64_t outer;                 // number of outer indices
  int nseg;
  int64_t seg_size[TN_MAX_SEG];
  int64_t seg_sA[TN_MAX_SEG];
  int64_t seg_sB[TN_MAX_SEG];    // 0 for M legs (B does not have them)
  int64_t seg_sC[TN_MAX_SEG];
  int Ks, Ns;
  int hasB;                      // 0: unary reduction, B == tropical one (0)
  int64_t kA[TN_GATE_MAX_K];
  int64_t kB[TN_GATE_MAX_K];
  int64_t nB[TN_GATE_MAX_N];
  int64_t nC[TN_GATE_MAX_N];
  // counting planes: element distance between residue planes of each tensor
  int64_t planeA, planeB, planeC;
  int P;                          // residue planes (0 = values only)
};

// Strided batched max-plus GEMM: C[b, m, n] = max_k A[b, m, k] + B[b, k, n].
struct GemmParams {
  int64_t batch, M, N, K;
  int64_t sAb, sAm, sAk;
  int64_t sBb, sBk, sBn;
  int64_t sCb, sCm, sCn;
  int64_t planeA, planeB, planeC;
  int P;
};

// out[i_0, ..., i_{r-1}] (row-major over dims) = in[sum_j i_j * sin_j]
struct PermParams {
  int r;
  int64_t total;
  int64_t dims[TN_MAX_RANK];
  int64_t sin[TN_MAX_RANK];
  int64_t planeIn, planeOut;
  int P;
};

// One leaf tensor built from the couplings (Sec. II bond / vertex tensors).
// Legs are (u, v) with u < v, u the slower index.
struct LeafDesc {
  int64_t off_x;     // byte offset of the leaf's values in the arena
  int64_t off_n;     // byte offset of its residue plane 0 (counting only)
  int64_t plane;     // elements between residue planes
  int32_t kind;      // 0: bond (legs u, v), 1: isolated spin (leg u)
  int32_t edge;      // edge id (kind 0)
  int32_t u, v;      // spins
  int32_t fu, fv;    // 1: the field of u (v) is absorbed into this leaf
};

// One step of the argmax traceback (Sec. III): the step C = A (.) B whose
// output index is already fixed picks the first k maximising A + B and
// assigns the contracted spins.
struct TraceStep {
  int64_t offA, offB;          // element offsets (offB < 0: unary, B == 0)
  int32_t nfa, nfb, nk;        // fixed legs of A, of B; contracted legs
  int32_t Ks;                  // q^nk
  int32_t fa_spin[TN_MAX_TRACE_LEGS];
  int32_t fb_spin[TN_MAX_TRACE_LEGS];
  int64_t fa_stride[TN_MAX_TRACE_LEGS];
  int64_t fb_stride[TN_MAX_TRACE_LEGS];
  int32_t k_spin[TN_MAX_TRACE_LEGS];
  int64_t k_sA[TN_MAX_TRACE_LEGS];
  int64_t k_sB[TN_MAX_TRACE_LEGS];
};

// 61-bit pseudo-Mersenne primes p = 2^61 - c (reduction after Crandall).
struct PrimeSet {
  uint64_t c[TN_MAX_PRIMES];
};
