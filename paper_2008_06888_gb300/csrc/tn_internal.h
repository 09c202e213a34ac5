// tn_internal.h -- structures shared by the host planner/executor and the
// CUDA kernels of libtn.so.  Not part of the public ABI (include/tn.h).
#pragma once
#ifdef __CUDACC_RTC__
// runtime-compiled chain kernels: no C library headers
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
#else
#include <stdint.h>
#endif

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
  int32_t seg_sh[TN_MAX_SEG];    // log2(seg_size) when every size is a power of two, else -1
  int Ks, Ns;
  int hasB;                      // 0: unary reduction, B == tropical one (0)
  int unitB;                     // every count of B is 1: ties only add counts
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
  int rbytes;        // bytes of one residue (8, or 4 for 31-bit primes)
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
  int32_t chain;               // >= 0: this record is ChainTrace[chain]
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

// ---- fused gate chains
// A chain applies G consecutive rank-preserving gate contractions to one big
// tensor in a single pass: the tensor is cut into tiles over a set of t
// "local" legs (the q^w fastest legs, for coalescing, plus every leg a gate
// touches); each CTA loads a tile into shared memory, applies the gates in
// order and writes it back.  A replace gate contracts the leg at local stride
// ls and puts the new leg in its place: C[.., v, ..] = max_u A[.., u, ..] +
// B[u, v, b..]; a diagonal gate adds B[b..] (all of B's legs are legs of A).
#define TN_CHAIN_MAX_G 20
#define TN_CHAIN_MAX_T 12
#define TN_CHAIN_MAX_HI 128

struct ChainGate {
  int32_t kind;      // 0 replace, 1 diagonal, 2 contract (folded register chains, last)
  int32_t ls;        // local stride of the replaced leg (replace)
  int32_t nb;        // B legs that are legs of the tile (0..2)
  int32_t lsb[2];    // their local strides
  int32_t kspin;     // contracted spin (replace), for the traceback
  int32_t lsh;       // log2(ls) when q == 2
  int32_t lsbh[2];   // log2(lsb) when q == 2
  int32_t lrank[2];  // register chains: bit of a fixed leg in the outer index tau
  int32_t nBel;      // elements of B
  int32_t unitB;     // 1: every count of B is 1 (a leaf), ties only add counts
  int64_t offB;      // element offset of B's values in the arena
  int64_t offBn;     // u64 offset of B's residue plane 0 in the arena (counting)
  int64_t planeB;    // elements between B's residue planes
  int64_t sBk, sBn;  // B strides of the contracted and of the new leg
  int64_t sBb[2];    // B strides of the tile legs
};

// Folded register-chain gate (q = 2, values only).  Every diagonal gate that
// shares a leg with a replace gate of the same chain is added into that
// replace gate's operand (a term that does not depend on the eliminated digit
// commutes with the max), so a chain becomes a short list of table gates.
// A table gate reads one table of 8 << nf values:
//   index bit 0: contracted digit x (replace) / register leg J (diagonal)
//   index bit 1: new digit x'       (replace) / register leg K (diagonal)
//   index bit 2: register leg K     (replace; 0 when K < 0)
//   index bits 3..: digits of the fixed legs, (tau >> fsh[i]) & 1 (tau: the
//                   thread's outer index, its bits the outer legs, fastest first)
// The table is the sum of its components: component c is original gate
// cg[c]'s operand B, read at the offset sum over its legs l (contracted,
// new, tile leg 0, tile leg 1) of digit(index bit cbit[c][l]) * stride(l).
#define TN_TG_MAXC 8
#define TN_TG_MAXF 3
#define TN_TG_TABLE 64       // largest table (8 << TN_TG_MAXF values)
struct TGate {
  int8_t kind;                  // 0 replace, 1 diagonal, 2 contract (last; no new digit)
  int8_t J, K;                  // register legs (-1: none)
  int8_t nf, ncomp;
  int8_t fsh[TN_TG_MAXF];       // fixed legs: their bits in the outer index tau
  int8_t cg[TN_TG_MAXC];        // original gate of each component
  int8_t cbit[TN_TG_MAXC][4];   // table bit of each of its legs (-1: absent)
  int16_t code;                 // kernel dispatch code of (kind, J, K)
  int16_t toff;                 // table offset (values) in shared memory
  int32_t kspin;                // replace: contracted spin (traceback)
};

// mode 1 (q = 2 only, "register chains"): every thread owns the 2^t elements
// that differ in the chain's replaced legs (the register legs; t = RB); the
// replace gate's ls is a register-bit index, a B leg is a register bit
// (lsb >= 0) or a leg fixed per thread (lsb < 0, digit = (base >> lsbh) & 1);
// hi_off[e] is the state offset of register index e, seg_* decode the thread
// index over the other legs.
struct ChainParams {
  int32_t mode;            // 0: shared-memory tiles, 1: register chains
  int32_t q, t, tile;      // tile = q^t elements
  int32_t lo, nhi;         // tile = nhi * lo; lo = q^w contiguous elements
  int32_t loh;             // log2(lo) when q == 2
  int32_t nseg, ngates;
  int32_t P;               // residue planes (0 = values only)
  int64_t outer;           // number of tiles
  int64_t hi_off[TN_CHAIN_MAX_HI];
  int64_t seg_size[TN_MAX_SEG];
  int64_t seg_s[TN_MAX_SEG];
  int32_t seg_sh[TN_MAX_SEG];  // log2(seg_size) when q == 2
  int32_t seg_ssh[TN_MAX_SEG]; // log2(seg_s) when q == 2 (register chains)
  int64_t planeA, planeC;  // plane distances of input and output
  ChainGate g[TN_CHAIN_MAX_G];
  int32_t ntg;             // folded table gates (mode 1, P == 0); 0: use g[]
  int32_t ttotal;          // values of all their tables
  TGate tg[TN_CHAIN_MAX_G];
  // folded register chains: offsets of register state e in the input and in the
  // output tensor, and each outer segment's shift in both (hi_off / seg_ssh
  // describe the state between the gates)
  int64_t hi_in[TN_CHAIN_MAX_HI], hi_out[TN_CHAIN_MAX_HI];
  int32_t ssh_in[TN_MAX_SEG], ssh_out[TN_MAX_SEG];
};

// Traceback record of a chain: the tile of the chain input selected by the
// (already fixed) spins on the outer legs is recomputed gate by gate in
// shared memory, then walked backwards to fix each contracted spin.
struct ChainTrace {
  int64_t offIn;                       // element offset of the chain input
  int32_t nout;                        // outer legs
  int32_t out_spin[TN_MAX_TRACE_LEGS];
  int64_t out_stride[TN_MAX_TRACE_LEGS];
  int32_t local_spin[TN_CHAIN_MAX_T];  // spin on each local leg after the chain (slowest first)
  int32_t out_rank[TN_MAX_TRACE_LEGS]; // folded register chains: bit of each outer leg in tau
  ChainParams p;
};

// 61-bit pseudo-Mersenne primes p = 2^61 - c (reduction after Crandall), or,
// for counts run one prime per pass in 4-byte planes, 31-bit ones 2^31 - c.
struct PrimeSet {
  uint64_t c[TN_MAX_PRIMES];
  int32_t r32;   // 1: residue planes hold uint32 residues of primes 2^31 - c
};
