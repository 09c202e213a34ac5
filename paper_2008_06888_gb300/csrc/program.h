// program.h -- lowering of a classified contraction plan to a fixed sequence
// of kernel launches with statically planned arena offsets.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.h"
#include "planner.h"
#include "tn_internal.h"

namespace tn {

// Location of a tensor: byte offsets inside a buffer (values at xoff, residue
// plane 0 at noff, planes `plane` elements apart).
struct Loc {
  int buf = -1;
  int64_t xoff = 0, noff = 0, plane = 0;
};

struct BufInfo {
  int64_t bytes = 0;
  int first = 1 << 30, last = -1;
  int64_t off = -1;
};

enum OpKind { OP_LEAVES, OP_PERM, OP_GATE, OP_GEMM, OP_TRACE, OP_CHAIN };

struct Op {
  OpKind kind;
  Loc in0, in1, out;
  int idx = -1;              // into gates / gemms / perms
  int trace_begin = 0, trace_n = 0;
  double bytes = 0, macs = 0;  // algorithmic traffic and multiply-adds of the launch
};

enum ProgMode { PM_ENERGY = 0, PM_CONFIG = 1, PM_COUNT = 2 };

struct Program {
  ProgMode mode;
  Dtype dt;
  int q = 2, P = 0;
  int rbytes = 8;                    // bytes of one residue of the counting planes
  bool pass_prime = false;           // one 31-bit prime per pass: plane 0's prime is set per run
  std::vector<BufInfo> bufs;
  std::vector<Op> ops;
  std::vector<GateParams> gates;
  std::vector<GemmParams> gemms;
  std::vector<PermParams> perms;
  std::vector<ChainParams> chains;                  // fused gate chains
  std::vector<const void *> chain_jit;              // their compiled kernels (nullptr: interpreted)
  std::vector<std::vector<Loc>> chain_blocs;        // their gate operands
  std::vector<ChainTrace> chain_traces;             // traceback records of chains
  std::vector<Loc> ctrace_in;
  std::vector<std::vector<Loc>> ctrace_blocs;
  size_t trace_smem = 0;                            // dynamic smem of the trace kernel
  std::vector<LeafDesc> leaves;      // offsets absolute after planning
  std::vector<TraceStep> trace;      // offsets absolute after planning
  std::vector<Loc> traceA, traceB;
  Loc leaves_loc;
  std::vector<int64_t> leaf_elem;    // element offset of each leaf in the leaves buffer
  Loc root;
  int64_t arena_bytes = 0;
  int fwd_end = 0;                   // ops [0, fwd_end) are the forward pass
  int n_transposes = 0, n_gate = 0, n_gemm = 0, n_recompute = 0, n_chain = 0, n_chain_gates = 0;
  double macs = 0;                   // tropical multiply-adds of the forward steps
  // CUDA graphs of op ranges, captured on the second run of a range
  struct Graph {
    int begin, end, runs, B;
    const char *arena;
    const float *J, *h;
    const int8_t *state;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  // device copies (owned by the context)
  LeafDesc *d_leaves = nullptr;
  TraceStep *d_trace = nullptr;
  ChainTrace *d_chain_traces = nullptr;
};

// Build the program for a plan.  seg_bytes: traceback checkpoint segment
// budget (PM_CONFIG; <= 0 keeps every intermediate).
// rbytes: bytes of one residue of the counting planes (8: 61-bit primes; 4:
// 31-bit primes, the one-prime-per-pass counts).
bool build_program(const Net &net, const Plan &plan, ProgMode mode, Dtype dt, int P,
                   int64_t seg_bytes, Program *pr, std::string *err, int rbytes = 8);

int64_t abs_off(const Program &pr, const Loc &l);  // arena byte offset of values

}  // namespace tn
