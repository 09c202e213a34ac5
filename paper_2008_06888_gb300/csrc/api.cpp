// api.cpp -- the C ABI of include/tn.h: contexts, execution of the lowered
// programs on the device, and exact count reconstruction (CRT).
#include "../../include/tn.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "planner.h"
#include "program.h"
#include "jit.h"
#include "sampler.h"

using namespace tn;

// 61-bit primes p_i = 2^61 - c_i; the last one used by a call is the witness.
static const uint64_t kPrimeC[TN_MAX_PRIMES] = {1, 31, 45, 229, 259, 283, 339, 391, 403};
// 31-bit primes p_j = 2^31 - c_j of the one-prime-per-pass counts (4-byte
// planes): enough passes to cover 8 61-bit primes, plus a witness.
static const int kPasses31Max = 17;
static const uint64_t kPrime31C[kPasses31Max] = {1,   19,  61,  69,  85,  99,  105, 151, 159,
                                                 171, 225, 249, 295, 325, 379, 399, 411};

struct tn_ctx {
  Net net;
  Dtype dt = DT_F32;
  uint32_t flags = 0;
  bool ordered = false;
  Plan plan;
  std::string err;
  cudaStream_t stream = nullptr;
  bool dev_ready = false;
  int device = 0;
  float *d_J = nullptr, *d_h = nullptr;
  int32_t *d_eu = nullptr, *d_ev = nullptr;
  int8_t *d_state = nullptr, *d_out = nullptr;
  int *d_err = nullptr;
  bool couplings_dirty = true;
  char *d_arena = nullptr;
  int64_t arena_cap = 0;
  std::unique_ptr<Program> prog[3];
  int prog_P = 0, prog_rb = 8;
  bool have_state = false;
  bool fwd_done = false;   // tn_forward ran last; its checkpoints are live
  cudaStream_t cap_stream = nullptr;   // private stream for graph capture
  // measurement
  bool profiling = false;
  int64_t launches[7] = {0, 0, 0, 0, 0, 0, 0};
  double prof_ms[7] = {0, 0, 0, 0, 0, 0, 0}, prof_bytes[7] = {0, 0, 0, 0, 0, 0, 0};
  double prof_macs[7] = {0, 0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> ev_pool;
  struct Pending { int kind, e0, e1; };
  std::vector<Pending> pending;
  int ev_next = 0;
  // batch buffers (capacity bcap instances)
  int bcap = 0;
  float *d_Jb = nullptr, *d_hb = nullptr;
  int8_t *d_stateb = nullptr, *d_outb = nullptr;
  // host-side program of tn_energy_noalloc and the plan fingerprint it was built for
  std::unique_ptr<Program> prog_noalloc;
  uint64_t noalloc_fp = 0;
  // energies returned = e_scale * E_ising + e_offset (Max-2-SAT contexts: the
  // number of violated clauses; 1 and 0 otherwise)
  double e_scale = 1.0, e_offset = 0.0;
  bool host_couplings = true;   // net.J / net.h hold the couplings in use
  // counts one 31-bit prime per pass (4-byte planes): its program and the
  // prime of the pass in flight
  std::unique_ptr<Program> prog_pass;
  uint64_t pass_c = 1;
};

static std::string g_build_err;

namespace {

// NVTX range for profilers (no cost without an attached tool): every entry
// point that computes, every batch group and every eagerly launched op.
struct Nvtx {
  explicit Nvtx(const char *name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
  Nvtx(const Nvtx &) = delete;
  Nvtx &operator=(const Nvtx &) = delete;
};

const char *op_name(OpKind k) {
  switch (k) {
    case OP_LEAVES: return "leaves";
    case OP_PERM: return "transpose";
    case OP_GATE: return "gate";
    case OP_GEMM: return "maxplus_gemm";
    case OP_TRACE: return "traceback";
    case OP_CHAIN: return "gate_chain";
  }
  return "op";
}

tn_status fail(tn_ctx *c, tn_status s, const std::string &msg) {
  if (c) c->err = msg; else g_build_err = msg;
  return s;
}

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(ctx, TN_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool integral(const std::vector<float> &v) {
  for (float x : v)
    if (!(std::fabs(x) < (float)(1 << 20)) || std::nearbyint(x) != x) return false;
  return true;
}

int64_t env_i64(const char *name, int64_t dflt) {
  const char *s = std::getenv(name);
  if (!s || !*s) return dflt;
  return std::strtoll(s, nullptr, 10);
}

void free_program(Program *p) {
  if (!p) return;
  if (p->d_leaves) cudaFree(p->d_leaves);
  if (p->d_trace) cudaFree(p->d_trace);
  if (p->d_chain_traces) cudaFree(p->d_chain_traces);
  for (auto &g : p->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  p->graphs.clear();
  p->d_leaves = nullptr;
  p->d_trace = nullptr;
  p->d_chain_traces = nullptr;
}

tn_status ensure_device(tn_ctx *ctx) {
  if (!ctx->dev_ready) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
      return fail(ctx, TN_ECUDA, "no CUDA device available (there is no CPU fallback)");
    CK(cudaGetDevice(&ctx->device));
    const Net &n = ctx->net;
    CK(cudaMalloc(&ctx->d_J, std::max(1, n.m) * sizeof(float)));
    CK(cudaMalloc(&ctx->d_h, std::max(1, n.n) * sizeof(float)));
    CK(cudaMalloc(&ctx->d_eu, std::max(1, n.m) * sizeof(int32_t)));
    CK(cudaMalloc(&ctx->d_ev, std::max(1, n.m) * sizeof(int32_t)));
    CK(cudaMalloc(&ctx->d_state, std::max(1, n.n)));
    CK(cudaMalloc(&ctx->d_out, std::max(1, n.n)));
    CK(cudaMalloc(&ctx->d_err, sizeof(int)));
    CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
    if (n.m) {
      CK(cudaMemcpy(ctx->d_eu, n.eu.data(), n.m * sizeof(int32_t), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(ctx->d_ev, n.ev.data(), n.m * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    ctx->dev_ready = true;
    ctx->couplings_dirty = true;
  }
  if (ctx->couplings_dirty) {
    const Net &n = ctx->net;
    if (n.m)
      CK(cudaMemcpyAsync(ctx->d_J, n.J.data(), n.m * sizeof(float), cudaMemcpyHostToDevice,
                         ctx->stream));
    std::vector<float> h = n.h;
    if (h.empty()) h.assign(n.n, 0.f);
    CK(cudaMemcpyAsync(ctx->d_h, h.data(), n.n * sizeof(float), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->couplings_dirty = false;
  }
  return TN_OK;
}

tn_status get_program(tn_ctx *ctx, ProgMode mode, int P, Program **out, int rb = 8) {
  if (!ctx->ordered) return fail(ctx, TN_ESTATE, "tn_order has not been called");
  std::unique_ptr<Program> &slot = ctx->prog[mode];
  if (!slot || (mode == PM_COUNT && (ctx->prog_P != P || ctx->prog_rb != rb))) {
    if (slot) free_program(slot.get());
    slot.reset(new Program());
    int64_t seg = 0;
    if (mode == PM_CONFIG) {
      seg = env_i64("TN_CKPT_SEGMENT_BYTES", -1);
      if (seg < 0) {
        // keep everything when it fits in a quarter of the free memory,
        // otherwise segments of about sqrt(total * largest) bytes
        double total = 0, big = 0;
        for (auto &s : ctx->plan.steps) {
          double b = std::pow((double)ctx->net.q, (double)ctx->plan.legset[s.c].size()) * 4;
          total += b;
          big = std::max(big, b);
        }
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        seg = (total < 0.25 * (double)fr) ? 0 : (int64_t)std::max(2 * big, std::sqrt(total * big));
      }
    }
    std::string err;
    if (!build_program(ctx->net, ctx->plan, mode, ctx->dt, mode == PM_COUNT ? P : 0, seg,
                       slot.get(), &err, mode == PM_COUNT ? rb : 8)) {
      slot.reset();
      return fail(ctx, TN_EINVAL, err);
    }
    Program &p = *slot;
    if (!p.leaves.empty()) {
      CK(cudaMalloc(&p.d_leaves, p.leaves.size() * sizeof(LeafDesc)));
      CK(cudaMemcpy(p.d_leaves, p.leaves.data(), p.leaves.size() * sizeof(LeafDesc),
                    cudaMemcpyHostToDevice));
    }
    if (!p.trace.empty()) {
      CK(cudaMalloc(&p.d_trace, p.trace.size() * sizeof(TraceStep)));
      CK(cudaMemcpy(p.d_trace, p.trace.data(), p.trace.size() * sizeof(TraceStep),
                    cudaMemcpyHostToDevice));
    }
    if (!p.chain_traces.empty()) {
      CK(cudaMalloc(&p.d_chain_traces, p.chain_traces.size() * sizeof(ChainTrace)));
      CK(cudaMemcpy(p.d_chain_traces, p.chain_traces.data(),
                    p.chain_traces.size() * sizeof(ChainTrace), cudaMemcpyHostToDevice));
    }
    if (mode == PM_COUNT) {
      ctx->prog_P = P;
      ctx->prog_rb = rb;
    }
    // large value chains run as kernels compiled for their gate sequence; if
    // that fails they stay on the interpreting kernel (TN_JIT_STRICT: error)
    std::string jerr;
    if (!jit_chains(p.chains, p.dt, &p.chain_jit, &jerr)) {
      p.chain_jit.assign(p.chains.size(), nullptr);
      if (std::getenv("TN_JIT_STRICT")) return fail(ctx, TN_ECUDA, jerr);
    }
  }
  Program &p = *slot;
  if (p.arena_bytes > ctx->arena_cap) {
    if (ctx->d_arena) CK(cudaFree(ctx->d_arena));
    ctx->d_arena = nullptr;
    ctx->arena_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->d_arena, p.arena_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, TN_ENOMEM, "arena of " + std::to_string(p.arena_bytes) + " bytes: " +
                                      cudaGetErrorString(e));
    }
    ctx->arena_cap = p.arena_bytes;
  }
  *out = &p;
  return TN_OK;
}

cudaEvent_t next_event(tn_ctx *ctx) {
  if (ctx->ev_next == (int)ctx->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_pool[ctx->ev_next++];
}

void collect_profile(tn_ctx *ctx) {
  if (ctx->pending.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto &pd : ctx->pending) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev_pool[pd.e0], ctx->ev_pool[pd.e1]);
    ctx->prof_ms[pd.kind] += ms;
  }
  ctx->pending.clear();
  ctx->ev_next = 0;
}

int op_kind_slot(OpKind k) {
  switch (k) {
    case OP_LEAVES: return 0;
    case OP_PERM: return 1;
    case OP_GATE: return 2;
    case OP_GEMM: return 3;
    case OP_TRACE: return 4;
    case OP_CHAIN: return 6;
  }
  return 5;
}

// What one execution of a program range works on: B instances, their
// couplings and spin states.
struct RunArgs {
  Batch bt;
  const float *J = nullptr, *h = nullptr;
  int8_t *state = nullptr;
};

RunArgs single_args(tn_ctx *ctx) {
  RunArgs a;
  a.J = ctx->d_J;
  a.h = ctx->d_h;
  a.state = ctx->d_state;
  return a;
}

tn_status run_ops(tn_ctx *ctx, Program &p, int op_begin, int op_end, cudaStream_t st,
                  bool account, const RunArgs &ra) {
  char *ar = ctx->d_arena;
  const Batch &bt = ra.bt;
  PrimeSet ps;
  ps.r32 = p.rbytes == 4;
  for (int i = 0; i < TN_MAX_PRIMES; ++i) ps.c[i] = ps.r32 ? kPrime31C[i] : kPrimeC[i];
  if (p.pass_prime) ps.c[0] = ctx->pass_c;   // one 31-bit prime per pass
  auto X = [&](const Loc &l) -> void * { return l.buf < 0 ? nullptr : ar + abs_off(p, l); };
  auto Nn = [&](const Loc &l) -> uint64_t * {
    return l.buf < 0 ? nullptr : (uint64_t *)(ar + p.bufs[l.buf].off + l.noff);
  };
  if (p.mode == PM_CONFIG && op_end > p.fwd_end)
    CK(cudaMemsetAsync(ra.state, 0xff, (size_t)std::max(1, ctx->net.n) * bt.B, st));
  if (ctx->profiling && ctx->ev_next > 4096) collect_profile(ctx);
  for (int oi = op_begin; oi < op_end; ++oi) {
    const Op &op = p.ops[oi];
    cudaError_t e = cudaSuccess;
    const int slot = op_kind_slot(op.kind);
    Nvtx nv(op_name(op.kind));
    int e0 = -1;
    if (ctx->profiling) {
      e0 = ctx->ev_next;
      cudaEventRecord(next_event(ctx), st);
    }
    switch (op.kind) {
      case OP_LEAVES:
        e = launch_leaves(p.dt, p.q, p.d_leaves, (int)p.leaves.size(), ra.J, ra.h, ar, p.P,
                          p.rbytes, bt, st);
        break;
      case OP_PERM:
        e = launch_permute(p.perms[op.idx], X(op.in0), X(op.out), Nn(op.in0), Nn(op.out), bt, st);
        break;
      case OP_GATE:
        e = launch_gate(p.dt, p.gates[op.idx], X(op.in0), X(op.in1), X(op.out), Nn(op.in0),
                        Nn(op.in1), Nn(op.out), ps, bt, st);
        break;
      case OP_GEMM:
        e = launch_mpgemm(p.dt, p.gemms[op.idx], X(op.in0), X(op.in1), X(op.out), bt, st);
        if (e == cudaSuccess && p.P > 0)
          e = launch_gemm_count(p.dt, p.gemms[op.idx], X(op.in0), X(op.in1), X(op.out),
                                Nn(op.in0), Nn(op.in1), Nn(op.out), ps, bt, st);
        break;
      case OP_TRACE:
        e = launch_trace(p.dt, p.q, p.d_trace + op.trace_begin, op.trace_n, p.d_chain_traces,
                         p.trace_smem, ar, ra.state, ctx->net.n, ctx->d_err, bt, st);
        break;
      case OP_CHAIN:
        if (op.idx < (int)p.chain_jit.size() && p.chain_jit[op.idx])
          e = launch_jit_chain(p.chain_jit[op.idx], p.chains[op.idx], ar, X(op.in0), X(op.out), bt,
                               st);
        else
          e = launch_chain(p.dt, p.chains[op.idx], ar, X(op.in0), Nn(op.in0), X(op.out),
                           Nn(op.out), ps, bt, st);
        break;
    }
    if (e != cudaSuccess)
      return fail(ctx, TN_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    int nl = 1;
    if (op.kind == OP_GEMM && p.P > 0) nl = 2;
    if (op.kind == OP_PERM && p.P > 0) nl = 2;
    if (account) {
      ctx->launches[slot] += nl;
      ctx->prof_bytes[slot] += op.bytes * bt.B;
      ctx->prof_macs[slot] += op.macs * bt.B;
    }
    if (ctx->profiling) {
      int e1 = ctx->ev_next;
      cudaEventRecord(next_event(ctx), st);
      ctx->pending.push_back({slot, e0, e1});
    }
  }
  return TN_OK;
}

// launches are counted once per launch (a batched launch covers every
// instance); bytes and multiply-adds once per instance
void account_range(tn_ctx *ctx, const Program &p, int b, int e, int B) {
  for (int oi = b; oi < e; ++oi) {
    const Op &op = p.ops[oi];
    const int slot = op_kind_slot(op.kind);
    int nl = 1;
    if ((op.kind == OP_GEMM || op.kind == OP_PERM) && p.P > 0) nl = 2;
    ctx->launches[slot] += nl;
    ctx->prof_bytes[slot] += op.bytes * B;
    ctx->prof_macs[slot] += op.macs * B;
  }
}

// Eager on the first run of a range (and whenever profiling, or with
// TN_NO_GRAPH set); captured into a CUDA graph on the second run and
// replayed from then on.
tn_status run_program(tn_ctx *ctx, Program &p, int op_begin, int op_end, const RunArgs &ra) {
  if (op_end < 0) op_end = (int)p.ops.size();
  static const bool no_graph = std::getenv("TN_NO_GRAPH") != nullptr;
  if (ctx->profiling || no_graph || p.pass_prime)
    return run_ops(ctx, p, op_begin, op_end, ctx->stream, true, ra);
  Program::Graph *g = nullptr;
  for (auto &x : p.graphs)
    if (x.begin == op_begin && x.end == op_end && x.B == ra.bt.B && x.J == ra.J) g = &x;
  if (g && (g->arena != ctx->d_arena || g->state != ra.state || g->h != ra.h)) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    g->runs = 0;
    g->arena = ctx->d_arena;
    g->state = ra.state;
    g->h = ra.h;
  }
  if (!g) {
    Program::Graph ng{};
    ng.begin = op_begin;
    ng.end = op_end;
    ng.B = ra.bt.B;
    ng.arena = ctx->d_arena;
    ng.J = ra.J;
    ng.h = ra.h;
    ng.state = ra.state;
    p.graphs.push_back(ng);
    g = &p.graphs.back();
  }
  if (!g->exec && g->runs == 0) {
    g->runs = 1;
    return run_ops(ctx, p, op_begin, op_end, ctx->stream, true, ra);
  }
  if (!g->exec) {
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    tn_status s = run_ops(ctx, p, op_begin, op_end, ctx->cap_stream, false, ra);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (s != TN_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return fail(ctx, TN_ECUDA, std::string("graph capture: ") +
                                                       cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g->exec = nullptr;
      return fail(ctx, TN_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
  }
  CK(cudaGraphLaunch(g->exec, ctx->stream));
  g->runs++;
  account_range(ctx, p, op_begin, op_end, ra.bt.B);
  return TN_OK;
}

tn_status run_program(tn_ctx *ctx, Program &p, int op_begin = 0, int op_end = -1) {
  return run_program(ctx, p, op_begin, op_end, single_args(ctx));
}

double root_energy(const tn_ctx *ctx, const void *raw) {
  double E;
  if (ctx->dt == DT_F32) {
    float v;
    std::memcpy(&v, raw, 4);
    E = -(double)v;
  } else {
    int32_t v;
    std::memcpy(&v, raw, 4);
    E = -(double)v;
  }
  return ctx->e_scale * E + ctx->e_offset;
}

// ---- exact count from residues (Garner's mixed-radix CRT)
typedef unsigned __int128 u128;

uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }
uint64_t powmod_h(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod_h(r, a, p);
    a = mulmod_h(a, a, p);
    e >>= 1;
  }
  return r;
}

// limbs (little endian) <- value of residues r[0..P) mod primes p[0..P)
std::vector<uint64_t> crt(const std::vector<uint64_t> &r, const std::vector<uint64_t> &p) {
  const int P = (int)r.size();
  std::vector<uint64_t> c(P);
  for (int i = 0; i < P; ++i) {
    // c_i = (r_i - (c_0 + p_0 (c_1 + ...))) / (p_0 ... p_{i-1}) mod p_i
    uint64_t x = 0, prod = 1;
    for (int j = 0; j < i; ++j) {
      x = (x + mulmod_h(c[j] % p[i], prod, p[i])) % p[i];
      prod = mulmod_h(prod, p[j] % p[i], p[i]);
    }
    uint64_t d = (r[i] % p[i] + p[i] - x) % p[i];
    c[i] = mulmod_h(d, powmod_h(prod, p[i] - 2, p[i]), p[i]);
  }
  std::vector<uint64_t> v{0};
  for (int i = P - 1; i >= 0; --i) {
    // v = v * p_i + c_i
    u128 carry = c[i];
    for (auto &l : v) {
      u128 t = (u128)l * p[i] + carry;
      l = (uint64_t)t;
      carry = t >> 64;
    }
    if (carry) v.push_back((uint64_t)carry);
  }
  while (v.size() > 1 && v.back() == 0) v.pop_back();
  return v;
}

uint64_t limbs_mod(const std::vector<uint64_t> &v, uint64_t p) {
  u128 r = 0;
  for (int i = (int)v.size() - 1; i >= 0; --i) r = ((r << 64) | v[i]) % p;
  return (uint64_t)r;
}


// ---- batches of coupling sets on one context (same graph, same order)

int64_t batch_stride(const Program &p) { return (p.arena_bytes + 255) / 256 * 256; }

tn_status ensure_arena(tn_ctx *ctx, int64_t bytes) {
  if (bytes <= ctx->arena_cap) return TN_OK;
  if (ctx->d_arena) CK(cudaFree(ctx->d_arena));
  ctx->d_arena = nullptr;
  ctx->arena_cap = 0;
  cudaError_t e = cudaMalloc(&ctx->d_arena, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, TN_ENOMEM, "batch arena of " + std::to_string(bytes) + " bytes: " +
                                    cudaGetErrorString(e));
  }
  ctx->arena_cap = bytes;
  return TN_OK;
}

tn_status ensure_batch(tn_ctx *ctx, int B) {
  if (B <= ctx->bcap) return TN_OK;
  const Net &n = ctx->net;
  if (ctx->d_Jb) CK(cudaFree(ctx->d_Jb));
  if (ctx->d_hb) CK(cudaFree(ctx->d_hb));
  if (ctx->d_stateb) CK(cudaFree(ctx->d_stateb));
  if (ctx->d_outb) CK(cudaFree(ctx->d_outb));
  ctx->d_Jb = nullptr;
  ctx->d_hb = nullptr;
  ctx->d_stateb = ctx->d_outb = nullptr;
  ctx->bcap = 0;
  CK(cudaMalloc(&ctx->d_Jb, (size_t)B * std::max(1, n.m) * sizeof(float)));
  CK(cudaMalloc(&ctx->d_hb, (size_t)B * std::max(1, n.n) * sizeof(float)));
  CK(cudaMalloc(&ctx->d_stateb, (size_t)B * std::max(1, n.n)));
  CK(cudaMalloc(&ctx->d_outb, (size_t)B * std::max(1, n.n)));
  ctx->bcap = B;
  return TN_OK;
}

tn_status batch_setup(tn_ctx *ctx, int B, const float *J, const float *h, int on_device,
                      ProgMode mode, int P, Program **out, RunArgs *ra, int rb = 8) {
  const Net &n = ctx->net;
  if (B < 1) return fail(ctx, TN_EINVAL, "batch size must be >= 1");
  if (n.m > 0 && !J) return fail(ctx, TN_EINVAL, "J is NULL");
  const bool fields = !n.h.empty();
  if (fields && !h) return fail(ctx, TN_EINVAL, "the instance has fields: h is required");
  if (!fields && h) return fail(ctx, TN_EINVAL, "the instance was built without fields");
  if (!on_device && ctx->dt == DT_I32) {
    for (int64_t i = 0; i < (int64_t)B * n.m; ++i)
      if (std::nearbyint(J[i]) != J[i] || !(std::fabs(J[i]) < (float)(1 << 20)))
        return fail(ctx, TN_EINVAL, "INT32 context needs integral J");
    if (h)
      for (int64_t i = 0; i < (int64_t)B * n.n; ++i)
        if (std::nearbyint(h[i]) != h[i] || !(std::fabs(h[i]) < (float)(1 << 20)))
          return fail(ctx, TN_EINVAL, "INT32 context needs integral h");
  }
  tn_status s = ensure_device(ctx);
  if (s != TN_OK) return s;
  Program *p;
  if ((s = get_program(ctx, mode, P, &p, rb)) != TN_OK) return s;
  const int64_t stride = batch_stride(*p);
  if ((s = ensure_arena(ctx, stride * B)) != TN_OK) return s;
  if ((s = ensure_batch(ctx, B)) != TN_OK) return s;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n.m) CK(cudaMemcpyAsync(ctx->d_Jb, J, (size_t)B * n.m * sizeof(float), kind, ctx->stream));
  if (h) CK(cudaMemcpyAsync(ctx->d_hb, h, (size_t)B * n.n * sizeof(float), kind, ctx->stream));
  ctx->fwd_done = false;
  ra->bt.B = B;
  ra->bt.ib = stride;
  ra->bt.jstride = n.m;
  ra->bt.hstride = n.n;
  ra->J = ctx->d_Jb;
  ra->h = ctx->d_hb;
  ra->state = ctx->d_stateb;
  *out = p;
  return TN_OK;
}

// values (4 bytes each) of the root of every instance
tn_status batch_roots(tn_ctx *ctx, const Program &p, int B, std::vector<char> *raw) {
  raw->assign((size_t)B * 4, 0);
  CK(cudaMemcpy2DAsync(raw->data(), 4, ctx->d_arena + abs_off(p, p.root), batch_stride(p), 4, B,
                       cudaMemcpyDeviceToHost, ctx->stream));
  return TN_OK;
}

tn_status check_trace_err(tn_ctx *ctx) {
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (herr) {
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    return fail(ctx, TN_EINVAL, "traceback met an unassigned spin (internal planning error)");
  }
  return TN_OK;
}

// exact count of one instance from its residues (the last one is the witness)
// Residue planes that carry the range of n 61-bit primes (plus a witness):
// ceil(61 n / 31) 31-bit primes in 4-byte planes when they fit in
// TN_MAX_PRIMES planes (half the bytes per residue and a cheaper modular
// product), else n 61-bit primes in 8-byte planes.  TN_COUNT_61 forces the
// latter.
struct CountRep {
  int P, rb;
  std::vector<uint64_t> primes;   // P primes, the last the witness
};
CountRep count_rep(int n_primes) {
  CountRep r;
  const int n31 = (61 * n_primes + 30) / 31;
  if (n31 + 1 <= TN_MAX_PRIMES && std::getenv("TN_COUNT_61") == nullptr) {
    r.P = n31 + 1;
    r.rb = 4;
    for (int i = 0; i < r.P; ++i) r.primes.push_back((1ull << 31) - kPrime31C[i]);
  } else {
    r.P = n_primes + 1;
    r.rb = 8;
    for (int i = 0; i < r.P; ++i) r.primes.push_back((1ull << 61) - kPrimeC[i]);
  }
  return r;
}

// exact count from residues res[i] modulo rep.primes[i] (the last one the witness)
tn_status count_from_residues(tn_ctx *ctx, const std::vector<uint64_t> &res, const CountRep &rep,
                              std::vector<uint64_t> *v) {
  const size_t n = rep.primes.size() - 1;
  std::vector<uint64_t> r(res.begin(), res.begin() + n), pr(rep.primes.begin(), rep.primes.begin() + n);
  *v = crt(r, pr);
  if (limbs_mod(*v, rep.primes[n]) != res[n])
    return fail(ctx, TN_EOVERFLOW, "count exceeds the product of the primes (witness mismatch)");
  return TN_OK;
}

tn_status finish_count(tn_ctx *ctx, const std::vector<uint64_t> &res,
                       const std::vector<uint64_t> &pr, uint64_t *limbs, int32_t *n_limbs,
                       double *ln_count);
tn_status count_in_passes(tn_ctx *ctx, int n_primes, uint64_t *limbs, int32_t *n_limbs,
                          double *ln_count, double *E);

}  // namespace

extern "C" {

tn_status tn_build(tn_ctx **out, int32_t n_spins, int32_t n_edges, const int32_t *edges,
                   const float *J, const float *h, int32_t q, uint32_t flags) {
  tn_ctx *ctx = nullptr;
  if (!out) return fail(nullptr, TN_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_spins < 1 || n_edges < 0) return fail(nullptr, TN_EINVAL, "bad sizes");
  if (q != 2 && q != 3) return fail(nullptr, TN_EINVAL, "q must be 2 or 3");
  if (q == 3 && h) return fail(nullptr, TN_EINVAL, "fields are Ising only (q == 2)");
  if (n_edges > 0 && (!edges || !J)) return fail(nullptr, TN_EINVAL, "edges / J missing");
  std::unique_ptr<tn_ctx> c(new (std::nothrow) tn_ctx());
  if (!c) return fail(nullptr, TN_ENOMEM, "host allocation");
  Net &n = c->net;
  n.n = n_spins;
  n.q = q;
  n.m = n_edges;
  std::vector<std::pair<int, int>> seen;
  for (int e = 0; e < n_edges; ++e) {
    int u = edges[2 * e], v = edges[2 * e + 1];
    if (u < 0 || v < 0 || u >= n_spins || v >= n_spins || u == v)
      return fail(nullptr, TN_EINVAL, "edge " + std::to_string(e) + " has a bad spin id");
    n.eu.push_back(u);
    n.ev.push_back(v);
    n.J.push_back(J[e]);
    seen.push_back({std::min(u, v), std::max(u, v)});
  }
  std::sort(seen.begin(), seen.end());
  for (size_t i = 1; i < seen.size(); ++i)
    if (seen[i] == seen[i - 1]) return fail(nullptr, TN_EINVAL, "repeated edge");
  if (h) n.h.assign(h, h + n_spins);
  for (float x : n.J) if (!std::isfinite(x)) return fail(nullptr, TN_EINVAL, "J not finite");
  for (float x : n.h) if (!std::isfinite(x)) return fail(nullptr, TN_EINVAL, "h not finite");
  n.build_leaves();
  uint32_t dtf = flags & TN_DTYPE_MASK;
  bool integ = integral(n.J) && integral(n.h);
  if (dtf == TN_DTYPE_I32 && !integ) return fail(nullptr, TN_EINVAL, "INT32 needs integral J, h");
  c->dt = (dtf == TN_DTYPE_I32 || (dtf == TN_DTYPE_AUTO && integ)) ? DT_I32 : DT_F32;
  c->flags = flags;
  *out = c.release();
  return TN_OK;
}

tn_status tn_max2sat_couplings(int32_t n_vars, int32_t n_clauses, const int32_t *lits,
                               int32_t *n_edges, int32_t *edges, float *J, float *h) {
  if (n_vars < 1 || n_clauses < 0 || (n_clauses > 0 && !lits) || !n_edges || !h ||
      (n_clauses > 0 && (!edges || !J)))
    return fail(nullptr, TN_EINVAL, "bad Max-2-SAT arguments");
  // 4 * [clause violated] = 1 + u_a s_a + u_b s_b + u_a u_b s_a s_b with
  // u = +1 for a negated literal (false at s = +1) and -1 otherwise, so
  // -4 * cost = -n_clauses + sum J s s + sum h s with J = -u_a u_b, h = -u.
  std::map<std::pair<int, int>, int> at;
  std::vector<int> hv(n_vars, 0);
  int ne = 0;
  for (int c = 0; c < n_clauses; ++c) {
    int la = lits[2 * c], lb = lits[2 * c + 1];
    int a = std::abs(la) - 1, b = std::abs(lb) - 1;
    if (la == 0 || lb == 0 || a >= n_vars || b >= n_vars || a == b)
      return fail(nullptr, TN_EINVAL, "clause " + std::to_string(c) + " has a bad literal");
    int ua = la < 0 ? 1 : -1, ub = lb < 0 ? 1 : -1;
    hv[a] -= ua;
    hv[b] -= ub;
    std::pair<int, int> key(std::min(a, b), std::max(a, b));
    auto it = at.find(key);
    if (it == at.end()) {
      at[key] = ne;
      edges[2 * ne] = a;
      edges[2 * ne + 1] = b;
      J[ne] = (float)(-ua * ub);
      ++ne;
    } else {
      J[it->second] += (float)(-ua * ub);
    }
  }
  for (int i = 0; i < n_vars; ++i) h[i] = (float)hv[i];
  *n_edges = ne;
  return TN_OK;
}

tn_status tn_build_max2sat(tn_ctx **out, int32_t n_vars, int32_t n_clauses, const int32_t *lits,
                           uint32_t flags) {
  if (!out) return fail(nullptr, TN_EINVAL, "out is NULL");
  *out = nullptr;
  if ((flags & TN_DTYPE_MASK) == TN_DTYPE_F32)
    return fail(nullptr, TN_EINVAL, "Max-2-SAT contexts are integral (INT32)");
  if (n_vars < 1 || n_clauses < 0) return fail(nullptr, TN_EINVAL, "bad sizes");
  std::vector<int32_t> edges(2 * (size_t)std::max(n_clauses, 1));
  std::vector<float> J(std::max(n_clauses, 1)), h(n_vars);
  int32_t ne = 0;
  tn_status s = tn_max2sat_couplings(n_vars, n_clauses, lits, &ne, edges.data(), J.data(),
                                     h.data());
  if (s != TN_OK) return s;
  tn_ctx *c = nullptr;
  s = tn_build(&c, n_vars, ne, edges.data(), J.data(), h.data(), 2,
               (flags & ~TN_DTYPE_MASK) | TN_DTYPE_I32);
  if (s != TN_OK) return s;
  c->e_scale = 0.25;
  c->e_offset = 0.25 * (double)n_clauses;
  *out = c;
  return TN_OK;
}

int32_t tn_leaf_count(const tn_ctx *ctx) { return ctx ? (int32_t)ctx->net.leaves.size() : 0; }

tn_status tn_order(tn_ctx *ctx, int32_t method, const int32_t *seq, int32_t seq_len,
                   uint64_t seed, int32_t restarts, double *log2_peak, double *log2_ops) {
  if (!ctx) return TN_EINVAL;
  Tree t;
  std::string err;
  bool ok = false;
  if (method == TN_ORDER_SWEEP) {
    std::vector<int> s;
    if (seq_len > 0 && !seq) return fail(ctx, TN_EINVAL, "sweep: seq is NULL");
    for (int i = 0; i < seq_len; ++i) s.push_back(seq[i]);
    ok = tree_from_sweep(ctx->net, s, &t, &err);
  } else if (method == TN_ORDER_GREEDY) {
    CostModel cm;
    // rank candidates by their lowered (fused) energy program on GB300 rates
    Dtype dt = ctx->dt;
    auto score = [&](const Plan &pl) -> double {
      Program pg;
      std::string e2;
      if (!build_program(ctx->net, pl, PM_ENERGY, dt, 0, 0, &pg, &e2)) return INFINITY;
      double tsec = 0;
      for (const Op &op : pg.ops) {
        tsec += 2.0e-6;  // launch / latency floor per kernel in a graph
        if (op.kind == OP_CHAIN) tsec += op.bytes / 3.4e12;
        else if (op.kind == OP_GEMM) tsec += std::max(op.macs / 1.2e13, op.bytes / 3.0e12);
        else tsec += op.bytes / 2.5e12;
      }
      return tsec;
    };
    ok = tree_greedy(ctx->net, seed, restarts, cm, &t, &err,
                     std::getenv("TN_GREEDY_STEP_COST") ? nullptr : std::function<double(const Plan &)>(score));
  } else if (method == TN_ORDER_TREE) {
    if (seq_len % 2 || (seq_len > 0 && !seq)) return fail(ctx, TN_EINVAL, "tree: odd length");
    for (int i = 0; i < seq_len; i += 2) t.steps.push_back({seq[i], seq[i + 1]});
    ok = true;
  } else {
    return fail(ctx, TN_EINVAL, "unknown order method");
  }
  if (!ok) return fail(ctx, TN_EINVAL, err);
  Plan p;
  if (!classify(ctx->net, t, &p, &err)) return fail(ctx, TN_EINVAL, err);
  if (p.log2_peak > 34.0) return fail(ctx, TN_ENOMEM, "largest tensor above 2^34 elements");
  for (auto &pg : ctx->prog) {
    if (pg) free_program(pg.get());
    pg.reset();
  }
  if (ctx->prog_pass) free_program(ctx->prog_pass.get());
  ctx->prog_pass.reset();
  ctx->plan = p;
  ctx->ordered = true;
  ctx->have_state = false;
  if (log2_peak) *log2_peak = p.log2_peak;
  if (log2_ops) *log2_ops = p.log2_ops;
  return TN_OK;
}

tn_status tn_set_couplings(tn_ctx *ctx, const float *J, const float *h, int32_t on_device) {
  if (!ctx) return TN_EINVAL;
  Net &n = ctx->net;
  if (h && n.q != 2) return fail(ctx, TN_EINVAL, "fields are Ising only");
  if (h && n.h.empty()) return fail(ctx, TN_EINVAL, "instance was built without fields");
  if (!on_device) {
    std::vector<float> nj(J ? J : n.J.data(), (J ? J : n.J.data()) + n.m);
    std::vector<float> nh = n.h;
    if (h) nh.assign(h, h + n.n);
    if (ctx->dt == DT_I32 && !(integral(nj) && integral(nh)))
      return fail(ctx, TN_EINVAL, "INT32 context needs integral J, h");
    n.J = nj;
    n.h = nh;
    ctx->couplings_dirty = true;
    ctx->host_couplings = true;
    return TN_OK;
  }
  tn_status s = ensure_device(ctx);
  ctx->host_couplings = false;
  if (s != TN_OK) return s;
  if (J && n.m)
    CK(cudaMemcpyAsync(ctx->d_J, J, n.m * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  if (h) CK(cudaMemcpyAsync(ctx->d_h, h, n.n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  return TN_OK;
}

tn_status tn_set_stream(tn_ctx *ctx, void *cuda_stream) {
  if (!ctx) return TN_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return TN_OK;
}

tn_status tn_energy(tn_ctx *ctx, double *E) {
  Nvtx nv("tn_energy");
  if (!ctx || !E) return fail(ctx, TN_EINVAL, "NULL argument");
  ctx->fwd_done = false;
  tn_status s = ensure_device(ctx);
  if (s != TN_OK) return s;
  Program *p;
  if ((s = get_program(ctx, PM_ENERGY, 0, &p)) != TN_OK) return s;
  if ((s = run_program(ctx, *p)) != TN_OK) return s;
  char raw[4];
  CK(cudaMemcpyAsync(raw, ctx->d_arena + abs_off(*p, p->root), 4, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *E = root_energy(ctx, raw);
  return TN_OK;
}

tn_status tn_forward(tn_ctx *ctx, double *E) {
  Nvtx nv("tn_forward");
  if (!ctx) return TN_EINVAL;
  tn_status s = ensure_device(ctx);
  if (s != TN_OK) return s;
  Program *p;
  if ((s = get_program(ctx, PM_CONFIG, 0, &p)) != TN_OK) return s;
  ctx->fwd_done = false;
  if ((s = run_program(ctx, *p, 0, p->fwd_end)) != TN_OK) return s;
  if (E) {
    char raw[4];
    CK(cudaMemcpyAsync(raw, ctx->d_arena + abs_off(*p, p->root), 4, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *E = root_energy(ctx, raw);
  }
  ctx->fwd_done = true;
  return TN_OK;
}

tn_status tn_backward(tn_ctx *ctx, int8_t *sigma) {
  Nvtx nv("tn_backward");
  if (!ctx) return TN_EINVAL;
  if (!ctx->fwd_done || !ctx->prog[PM_CONFIG])
    return fail(ctx, TN_ESTATE, "tn_backward needs tn_forward as the previous call");
  Program &p = *ctx->prog[PM_CONFIG];
  tn_status s;
  ctx->fwd_done = false;
  if ((s = run_program(ctx, p, p.fwd_end, (int)p.ops.size())) != TN_OK) return s;
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (herr) {
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    return fail(ctx, TN_EINVAL, "traceback met an unassigned spin (internal planning error)");
  }
  ctx->have_state = true;
  if (sigma) {
    CK(launch_state_out(ctx->net.q, ctx->net.n, ctx->d_state, ctx->d_out, 1, ctx->stream));
    ctx->launches[5]++;
    CK(cudaMemcpyAsync(sigma, ctx->d_out, ctx->net.n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return TN_OK;
}

tn_status tn_config(tn_ctx *ctx, int8_t *sigma, double *E) {
  tn_status s = tn_forward(ctx, E);
  if (s != TN_OK) return s;
  return tn_backward(ctx, sigma);
}

tn_status tn_gradient(tn_ctx *ctx, float *dJ, float *dh, int32_t on_device) {
  if (!ctx) return TN_EINVAL;
  if (ctx->e_scale != 1.0) return fail(ctx, TN_ESTATE, "no coupling gradient for Max-2-SAT");
  if (!ctx->have_state) return fail(ctx, TN_ESTATE, "tn_config has not run");
  const Net &n = ctx->net;
  if (on_device) {
    CK(launch_grad(n.q, n.n, n.m, ctx->d_eu, ctx->d_ev, ctx->d_state, dJ, dh, 1, ctx->stream));
    return TN_OK;
  }
  float *gJ = nullptr, *gh = nullptr;
  CK(cudaMalloc(&gJ, std::max(1, n.m) * sizeof(float)));
  CK(cudaMalloc(&gh, std::max(1, n.n) * sizeof(float)));
  CK(launch_grad(n.q, n.n, n.m, ctx->d_eu, ctx->d_ev, ctx->d_state, gJ, gh, 1, ctx->stream));
  if (dJ && n.m) CK(cudaMemcpyAsync(dJ, gJ, n.m * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (dh) CK(cudaMemcpyAsync(dh, gh, n.n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  cudaFree(gJ);
  cudaFree(gh);
  return TN_OK;
}

tn_status tn_count(tn_ctx *ctx, int32_t n_primes, uint64_t *limbs, int32_t *n_limbs,
                   double *ln_count, double *E) {
  Nvtx nv("tn_count");
  if (!ctx) return TN_EINVAL;
  ctx->fwd_done = false;
  if (n_primes < 1 || n_primes > TN_MAX_PRIMES - 1)
    return fail(ctx, TN_EINVAL, "n_primes must be in [1, 8]");
  tn_status s = ensure_device(ctx);
  if (s != TN_OK) return s;
  const CountRep rep = count_rep(n_primes);
  Program *p;
  const bool force_passes = std::getenv("TN_COUNT_PASSES") != nullptr;
  if (force_passes) return count_in_passes(ctx, n_primes, limbs, n_limbs, ln_count, E);
  s = get_program(ctx, PM_COUNT, rep.P, &p, rep.rb);
  if (s == TN_ENOMEM) {
    // the residue planes do not fit: one 31-bit prime per pass
    if (ctx->prog[PM_COUNT]) free_program(ctx->prog[PM_COUNT].get());
    ctx->prog[PM_COUNT].reset();
    return count_in_passes(ctx, n_primes, limbs, n_limbs, ln_count, E);
  }
  if (s != TN_OK) return s;
  if ((s = run_program(ctx, *p)) != TN_OK) return s;
  char raw[4];
  std::vector<uint64_t> res(rep.P, 0);
  const char *base = ctx->d_arena + p->bufs[p->root.buf].off;
  CK(cudaMemcpyAsync(raw, base + p->root.xoff, 4, cudaMemcpyDeviceToHost, ctx->stream));
  for (int i = 0; i < rep.P; ++i)   // little-endian: a 4-byte residue fills the low half
    CK(cudaMemcpyAsync(&res[i], base + p->root.noff + (int64_t)i * p->root.plane * rep.rb, rep.rb,
                       cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (E) *E = root_energy(ctx, raw);
  return finish_count(ctx, res, rep.primes, limbs, n_limbs, ln_count);
}

}  // extern "C"

namespace {

// count from residues res[i] modulo primes pr[i], the last pair the witness
tn_status finish_count(tn_ctx *ctx, const std::vector<uint64_t> &res,
                       const std::vector<uint64_t> &pr, uint64_t *limbs, int32_t *n_limbs,
                       double *ln_count) {
  const size_t n = pr.size() - 1;
  std::vector<uint64_t> r(res.begin(), res.begin() + n), p(pr.begin(), pr.begin() + n);
  std::vector<uint64_t> v = crt(r, p);
  if (limbs_mod(v, pr[n]) != res[n])
    return fail(ctx, TN_EOVERFLOW, "count exceeds the product of the primes (witness mismatch)");
  if (n_limbs) {
    if (limbs && *n_limbs < (int32_t)v.size())
      return fail(ctx, TN_EINVAL, "limbs buffer too small");
    if (limbs) for (size_t i = 0; i < v.size(); ++i) limbs[i] = v[i];
    *n_limbs = (int32_t)v.size();
  }
  if (ln_count) {
    long double x = 0;
    for (int i = (int)v.size() - 1; i >= 0; --i) x = x * 18446744073709551616.0L + (long double)v[i];
    *ln_count = (double)std::log(x);
  }
  return TN_OK;
}

// The degeneracy with one 31-bit prime per pass: the program keeps a single
// 4-byte residue plane (values + 4 bytes per element instead of 4 + 8 (n + 1)),
// so instances whose planes for n 61-bit primes do not fit in device memory
// still count exactly.  Enough passes to reach the range of n 61-bit primes,
// then one witness pass; Garner's CRT over the pass residues on the host.
tn_status count_in_passes(tn_ctx *ctx, int n_primes, uint64_t *limbs, int32_t *n_limbs,
                          double *ln_count, double *E) {
  const int n31 = (61 * n_primes + 30) / 31;
  if (n31 + 1 > kPasses31Max) return fail(ctx, TN_EINVAL, "too many primes for counting passes");
  if (!ctx->ordered) return fail(ctx, TN_ESTATE, "tn_order has not been called");
  if (!ctx->prog_pass) {
    std::unique_ptr<Program> pg(new Program());
    std::string err;
    if (!build_program(ctx->net, ctx->plan, PM_COUNT, ctx->dt, 1, 0, pg.get(), &err, 4))
      return fail(ctx, TN_EINVAL, err);
    pg->pass_prime = true;
    if (!pg->leaves.empty()) {
      CK(cudaMalloc(&pg->d_leaves, pg->leaves.size() * sizeof(LeafDesc)));
      CK(cudaMemcpy(pg->d_leaves, pg->leaves.data(), pg->leaves.size() * sizeof(LeafDesc),
                    cudaMemcpyHostToDevice));
    }
    ctx->prog_pass = std::move(pg);
  }
  Program &p = *ctx->prog_pass;
  tn_status s = ensure_arena(ctx, p.arena_bytes);
  if (s != TN_OK) return s;
  std::vector<uint64_t> res(n31 + 1), pr(n31 + 1);
  char raw[4];
  for (int j = 0; j <= n31; ++j) {
    ctx->pass_c = kPrime31C[j];
    pr[j] = (1ull << 31) - kPrime31C[j];
    if ((s = run_program(ctx, p)) != TN_OK) return s;
    const char *base = ctx->d_arena + p.bufs[p.root.buf].off;
    uint32_t r = 0;
    if (j == 0) CK(cudaMemcpyAsync(raw, base + p.root.xoff, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&r, base + p.root.noff, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    res[j] = r;
  }
  if (E) *E = root_energy(ctx, raw);
  return finish_count(ctx, res, pr, limbs, n_limbs, ln_count);
}

}  // namespace

extern "C" {


tn_status tn_energy_batch(tn_ctx *ctx, int32_t B, const float *J, const float *h,
                          int32_t on_device, double *E) {
  Nvtx nv("tn_energy_batch");
  if (!ctx) return TN_EINVAL;
  if (!E) return fail(ctx, TN_EINVAL, "E is NULL");
  Program *p;
  RunArgs ra;
  tn_status s = batch_setup(ctx, B, J, h, on_device, PM_ENERGY, 0, &p, &ra);
  if (s != TN_OK) return s;
  if ((s = run_program(ctx, *p, 0, -1, ra)) != TN_OK) return s;
  std::vector<char> raw;
  if ((s = batch_roots(ctx, *p, B, &raw)) != TN_OK) return s;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int b = 0; b < B; ++b) E[b] = root_energy(ctx, raw.data() + 4 * b);
  return TN_OK;
}

tn_status tn_config_batch(tn_ctx *ctx, int32_t B, const float *J, const float *h,
                          int32_t on_device, double *E, int8_t *sigma) {
  Nvtx nv("tn_config_batch");
  if (!ctx) return TN_EINVAL;
  Program *p;
  RunArgs ra;
  tn_status s = batch_setup(ctx, B, J, h, on_device, PM_CONFIG, 0, &p, &ra);
  if (s != TN_OK) return s;
  if ((s = run_program(ctx, *p, 0, -1, ra)) != TN_OK) return s;
  std::vector<char> raw;
  if (E && (s = batch_roots(ctx, *p, B, &raw)) != TN_OK) return s;
  if (sigma) {
    CK(launch_state_out(ctx->net.q, ctx->net.n, ctx->d_stateb, ctx->d_outb, B, ctx->stream));
    ctx->launches[5]++;
    CK(cudaMemcpyAsync(sigma, ctx->d_outb, (size_t)B * ctx->net.n, cudaMemcpyDeviceToHost,
                       ctx->stream));
  }
  if ((s = check_trace_err(ctx)) != TN_OK) return s;
  if (E)
    for (int b = 0; b < B; ++b) E[b] = root_energy(ctx, raw.data() + 4 * b);
  return TN_OK;
}

}  // extern "C"

namespace {

// Non-blocking streams of tn_batch_run, created once per device.
constexpr int kBatchStreams = 4;
tn_status batch_streams(tn_ctx *ctx, std::vector<cudaStream_t> *out) {
  static std::mutex mu;
  static std::map<int, std::vector<cudaStream_t>> pools;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  std::vector<cudaStream_t> &v = pools[dev];
  while ((int)v.size() < kBatchStreams) {
    cudaStream_t st;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    v.push_back(st);
  }
  *out = v;
  return TN_OK;
}

// Pinned host staging of the calling thread (grown as needed, kept for reuse).
tn_status pinned_stage(tn_ctx *ctx, size_t bytes, char **out) {
  thread_local char *buf = nullptr;
  thread_local size_t cap = 0;
  if (bytes > cap) {
    if (buf) cudaFreeHost(buf);
    buf = nullptr;
    cap = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20);
    CK(cudaHostAlloc(reinterpret_cast<void **>(&buf), want, cudaHostAllocDefault));
    cap = want;
  }
  *out = buf;
  return TN_OK;
}

// E, counts and statuses of B instances from their staged root values (raw:
// 4 bytes each) and residues (res[i * B + b], plane i, the last the witness).
tn_status finish_counts(tn_ctx *ctx, int B, const CountRep &rep, const char *raw,
                        const uint64_t *res, uint64_t *limbs, int32_t limbs_per, double *E,
                        int32_t *status) {
  const int P = rep.P;
  tn_status first = TN_OK;
  for (int b = 0; b < B; ++b) {
    if (E) E[b] = root_energy(ctx, raw + 4 * b);
    std::vector<uint64_t> r(P), v;
    for (int i = 0; i < P; ++i) r[i] = res[(size_t)i * B + b];
    tn_status sb = count_from_residues(ctx, r, rep, &v);
    if (sb == TN_OK && (int)v.size() > limbs_per) {
      sb = TN_EINVAL;
      fail(ctx, sb, "limbs_per too small for a count");
    }
    uint64_t *out = limbs + (int64_t)b * limbs_per;
    for (int i = 0; i < limbs_per; ++i) out[i] = (sb == TN_OK && i < (int)v.size()) ? v[i] : 0;
    if (status) status[b] = sb;
    if (sb != TN_OK && first == TN_OK) first = sb;
  }
  return first;
}

// queue the copies of B roots (and P residue planes) of a program's batch to host
// staging; 4-byte residues land in the low halves of the (zeroed) 8-byte slots
tn_status stage_results(tn_ctx *ctx, const Program &p, int B, int P, char *raw, uint64_t *res) {
  CK(cudaMemcpy2DAsync(raw, 4, ctx->d_arena + abs_off(p, p.root), batch_stride(p), 4, B,
                       cudaMemcpyDeviceToHost, ctx->stream));
  const char *rbase = ctx->d_arena + p.bufs[p.root.buf].off + p.root.noff;
  const int rb = p.rbytes;
  if (rb != 8) std::memset(res, 0, (size_t)P * B * 8);
  for (int i = 0; i < P; ++i)
    CK(cudaMemcpy2DAsync(res + (size_t)i * B, 8, rbase + (int64_t)i * p.root.plane * rb,
                         batch_stride(p), rb, B, cudaMemcpyDeviceToHost, ctx->stream));
  return TN_OK;
}

}  // namespace

extern "C" {

tn_status tn_count_batch(tn_ctx *ctx, int32_t B, const float *J, const float *h,
                         int32_t on_device, int32_t n_primes, uint64_t *limbs, int32_t limbs_per,
                         double *E, int32_t *status) {
  Nvtx nv("tn_count_batch");
  if (!ctx) return TN_EINVAL;
  if (n_primes < 1 || n_primes > TN_MAX_PRIMES - 1)
    return fail(ctx, TN_EINVAL, "n_primes must be in [1, 8]");
  if (!limbs || limbs_per < 1) return fail(ctx, TN_EINVAL, "limbs buffer missing");
  const CountRep rep = count_rep(n_primes);
  const int P = rep.P;
  Program *p;
  RunArgs ra;
  tn_status s = batch_setup(ctx, B, J, h, on_device, PM_COUNT, P, &p, &ra, rep.rb);
  if (s != TN_OK) return s;
  if ((s = run_program(ctx, *p, 0, -1, ra)) != TN_OK) return s;
  std::vector<char> raw((size_t)B * 4);
  std::vector<uint64_t> res((size_t)P * B);
  if ((s = stage_results(ctx, *p, B, P, raw.data(), res.data())) != TN_OK) return s;
  CK(cudaStreamSynchronize(ctx->stream));
  return finish_counts(ctx, B, rep, raw.data(), res.data(), limbs, limbs_per, E, status);
}

tn_status tn_batch_run(int32_t B, tn_ctx *const *ctxs, double *E, uint64_t *limbs,
                       int32_t limbs_per, int32_t *status) {
  Nvtx nv("tn_batch_run");
  if (B < 0 || (B > 0 && !ctxs)) return TN_EINVAL;
  // group the contexts whose graph, dtype and plan coincide; each group runs
  // as one batch on its first context
  auto key = [](const tn_ctx *c) {
    uint64_t f = 1469598103934665603ull;
    auto mix = [&](uint64_t x) { f = (f ^ x) * 1099511628211ull; };
    mix((uint64_t)c->net.n);
    mix((uint64_t)c->net.q);
    mix((uint64_t)c->dt);
    mix((uint64_t)c->net.h.empty());
    uint64_t ab[2];
    std::memcpy(&ab[0], &c->e_scale, 8);
    std::memcpy(&ab[1], &c->e_offset, 8);
    mix(ab[0]);
    mix(ab[1]);
    for (int e = 0; e < c->net.m; ++e) mix(((uint64_t)c->net.eu[e] << 32) | (uint32_t)c->net.ev[e]);
    for (auto &st : c->plan.steps) mix(((uint64_t)(st.a + 7) << 40) ^ ((uint64_t)(st.b + 7) << 20) ^ (uint64_t)st.c);
    return f;
  };
  // the hash only buckets; a context joins a group only if its graph, dtype,
  // energy map and steps equal those of the group's first context exactly
  auto same = [](const tn_ctx *a, const tn_ctx *b) {
    const Net &x = a->net, &y = b->net;
    if (x.n != y.n || x.q != y.q || x.m != y.m || a->dt != b->dt ||
        x.h.empty() != y.h.empty() || a->e_scale != b->e_scale || a->e_offset != b->e_offset ||
        x.eu != y.eu || x.ev != y.ev || a->plan.n_leaves != b->plan.n_leaves ||
        a->plan.steps.size() != b->plan.steps.size())
      return false;
    for (size_t i = 0; i < a->plan.steps.size(); ++i) {
      const PStep &s = a->plan.steps[i], &t = b->plan.steps[i];
      if (s.a != t.a || s.b != t.b || s.c != t.c) return false;
    }
    return true;
  };
  std::map<uint64_t, std::vector<std::vector<int>>> buckets;
  for (int k = 0; k < B; ++k) {
    if (!ctxs[k] || !ctxs[k]->ordered) {
      if (status) status[k] = TN_ESTATE;
      continue;
    }
    std::vector<std::vector<int>> &bk = buckets[key(ctxs[k])];
    bool placed = false;
    for (auto &g : bk)
      if (same(ctxs[g[0]], ctxs[k])) {
        g.push_back(k);
        placed = true;
        break;
      }
    if (!placed) bk.push_back({k});
  }
  std::vector<std::vector<int>> groups;
  for (auto &kv : buckets)
    for (auto &g : kv.second) groups.push_back(std::move(g));
  tn_status first = TN_OK;
  for (int k = 0; k < B; ++k)
    if (!ctxs[k] || !ctxs[k]->ordered) first = TN_ESTATE;
  // Every group is queued before any is waited for: group g runs on stream
  // g mod kBatchStreams of a pool, largest groups first, so the small groups'
  // launch-bound steps overlap the large groups' bandwidth-bound ones; the
  // roots and residues land in pinned host staging, read after one wait.
  std::sort(groups.begin(), groups.end(), [&](const std::vector<int> &a, const std::vector<int> &b) {
    const double wa = a.size() * std::exp2(ctxs[a[0]]->plan.log2_peak);
    const double wb = b.size() * std::exp2(ctxs[b[0]]->plan.log2_peak);
    return wa > wb;
  });
  const CountRep rep = count_rep(3);   // the range of 3 61-bit primes + witness
  const int P = limbs ? rep.P : 0;
  size_t stage_bytes = 0;
  for (auto &ids : groups) stage_bytes += ids.size() * (4 + 8 * (size_t)P) + 64;
  char *stage = nullptr;
  std::vector<cudaStream_t> pool;
  tn_status ps_status = TN_OK;
  if (!groups.empty()) {
    tn_ctx *c0 = ctxs[groups[0][0]];
    ps_status = ensure_device(c0);
    if (ps_status == TN_OK) ps_status = batch_streams(c0, &pool);
    if (ps_status == TN_OK) ps_status = pinned_stage(c0, stage_bytes, &stage);
  }
  struct Run {
    tn_ctx *owner;
    cudaStream_t orig;
    Program *p = nullptr;
    char *raw = nullptr;
    uint64_t *res = nullptr;
    tn_status s = TN_OK;
  };
  std::vector<Run> runs(groups.size());
  size_t off = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::vector<int> &ids = groups[gi];
    Run &r = runs[gi];
    r.owner = ctxs[ids[0]];
    r.orig = r.owner->stream;
    if (ps_status != TN_OK) {
      r.s = ps_status;
      continue;
    }
    const Net &n = r.owner->net;
    const int G = (int)ids.size();
    r.res = reinterpret_cast<uint64_t *>(stage + off);
    off += (size_t)G * 8 * P;
    r.raw = stage + off;
    off += ((size_t)G * 4 + 63) / 64 * 64;
    std::vector<float> J((size_t)G * n.m), h(n.h.empty() ? 0 : (size_t)G * n.n);
    for (int g = 0; g < G; ++g) {
      const Net &ng = ctxs[ids[g]]->net;
      std::copy(ng.J.begin(), ng.J.end(), J.begin() + (size_t)g * n.m);
      if (!h.empty()) std::copy(ng.h.begin(), ng.h.end(), h.begin() + (size_t)g * n.n);
    }
    // the pool stream starts after the work already queued on the context's
    // stream; with profiling on, the groups share one stream so that the
    // per-launch event times do not include other groups' concurrent kernels
    bool prof = false;
    for (auto &g2 : groups) prof = prof || ctxs[g2[0]]->profiling;
    cudaStream_t st = pool[prof ? 0 : gi % pool.size()];
    if (cudaStreamSynchronize(r.orig) != cudaSuccess) {
      r.s = fail(r.owner, TN_ECUDA, "stream of a batch context failed");
      continue;
    }
    r.owner->stream = st;
    RunArgs ra;
    r.s = batch_setup(r.owner, G, J.data(), h.empty() ? nullptr : h.data(), 0,
                      limbs ? PM_COUNT : PM_ENERGY, P, &r.p, &ra, rep.rb);
    if (r.s == TN_OK) r.s = run_program(r.owner, *r.p, 0, -1, ra);
    if (r.s == TN_OK) r.s = stage_results(r.owner, *r.p, G, P, r.raw, r.res);
  }
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::vector<int> &ids = groups[gi];
    Run &r = runs[gi];
    const int G = (int)ids.size();
    if (r.owner->stream != r.orig) {
      tn_ctx *ctx = r.owner;
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      ctx->stream = r.orig;
      if (e != cudaSuccess && r.s == TN_OK)
        r.s = fail(ctx, TN_ECUDA, std::string("batch group: ") + cudaGetErrorString(e));
    }
    std::vector<double> Eg(G);
    std::vector<int32_t> sg(G, TN_OK);
    tn_status s = r.s;
    if (s == TN_OK && limbs) {
      std::vector<uint64_t> lg((size_t)G * limbs_per);
      s = finish_counts(r.owner, G, rep, r.raw, r.res, lg.data(), limbs_per, Eg.data(), sg.data());
      for (int g = 0; g < G; ++g)
        std::copy(lg.begin() + (size_t)g * limbs_per, lg.begin() + (size_t)(g + 1) * limbs_per,
                  limbs + (int64_t)ids[g] * limbs_per);
    } else if (s == TN_OK) {
      for (int g = 0; g < G; ++g) Eg[g] = root_energy(r.owner, r.raw + 4 * g);
    } else {
      std::fill(sg.begin(), sg.end(), s);
      if (limbs)
        for (int g = 0; g < G; ++g)
          std::fill(limbs + (int64_t)ids[g] * limbs_per, limbs + (int64_t)(ids[g] + 1) * limbs_per,
                    0ull);
    }
    if (s != TN_OK)
      for (int g = 0; g < G; ++g)
        if (sg[g] == TN_OK) sg[g] = s == TN_EOVERFLOW ? TN_OK : s;
    for (int g = 0; g < G; ++g) {
      if (E) E[ids[g]] = Eg[g];
      if (status) status[ids[g]] = sg[g];
      if (sg[g] != TN_OK && first == TN_OK) first = (tn_status)sg[g];
    }
  }
  return first;
}

tn_status tn_set_profiling(tn_ctx *ctx, int32_t enable) {
  if (!ctx) return TN_EINVAL;
  collect_profile(ctx);
  ctx->profiling = enable != 0;
  return TN_OK;
}

tn_status tn_profile_get(tn_ctx *ctx, int32_t kind, int64_t *launches, double *ms,
                         double *bytes, double *macs) {
  if (!ctx || kind < -1 || kind > 6) return TN_EINVAL;
  collect_profile(ctx);
  int64_t l = 0;
  double t = 0, b = 0, m = 0;
  for (int k = 0; k < 7; ++k)
    if (kind == -1 || kind == k) {
      l += ctx->launches[k];
      t += ctx->prof_ms[k];
      b += ctx->prof_bytes[k];
      m += ctx->prof_macs[k];
    }
  if (launches) *launches = l;
  if (ms) *ms = t;
  if (bytes) *bytes = b;
  if (macs) *macs = m;
  return TN_OK;
}

tn_status tn_profile_reset(tn_ctx *ctx) {
  if (!ctx) return TN_EINVAL;
  collect_profile(ctx);
  for (int k = 0; k < 7; ++k) {
    ctx->launches[k] = 0;
    ctx->prof_ms[k] = ctx->prof_bytes[k] = ctx->prof_macs[k] = 0;
  }
  return TN_OK;
}

tn_status tn_plan_info(const tn_ctx *ctx, int32_t *n_steps, int32_t *n_transposes,
                       int64_t *arena_energy, int64_t *arena_config, int64_t *arena_count) {
  if (!ctx) return TN_EINVAL;
  if (!ctx->ordered) return TN_ESTATE;
  Program pe, pc, pn;
  std::string err;
  if (n_steps) *n_steps = (int32_t)ctx->plan.steps.size();
  if (n_transposes || arena_energy) {
    if (!build_program(ctx->net, ctx->plan, PM_ENERGY, ctx->dt, 0, 0, &pe, &err)) return TN_EINVAL;
    if (n_transposes) *n_transposes = pe.n_transposes;
    if (arena_energy) *arena_energy = pe.arena_bytes;
  }
  if (arena_config) {
    if (!build_program(ctx->net, ctx->plan, PM_CONFIG, ctx->dt, 0, 0, &pc, &err)) return TN_EINVAL;
    *arena_config = pc.arena_bytes;
  }
  if (arena_count) {
    const CountRep rep = count_rep(3);
    if (!build_program(ctx->net, ctx->plan, PM_COUNT, ctx->dt, rep.P, 0, &pn, &err, rep.rb))
      return TN_EINVAL;
    *arena_count = pn.arena_bytes;
  }
  return TN_OK;
}

tn_status tn_plan_launches(const tn_ctx *ctx, int32_t mode, int64_t *counts) {
  if (!ctx || !counts || mode < 0 || mode > 2) return TN_EINVAL;
  if (!ctx->ordered) return TN_ESTATE;
  Program pg;
  std::string err;
  const ProgMode pm = mode == 0 ? PM_ENERGY : mode == 1 ? PM_CONFIG : PM_COUNT;
  const CountRep rep = count_rep(3);
  if (!build_program(ctx->net, ctx->plan, pm, ctx->dt, pm == PM_COUNT ? rep.P : 0, 0, &pg, &err,
                     pm == PM_COUNT ? rep.rb : 8))
    return TN_EINVAL;
  for (int k = 0; k < 7; ++k) counts[k] = 0;
  for (const Op &op : pg.ops) {
    const int nl = ((op.kind == OP_GEMM || op.kind == OP_PERM) && pg.P > 0) ? 2 : 1;
    counts[op_kind_slot(op.kind)] += nl;
  }
  return TN_OK;
}

// For callers that cannot allocate device memory (see tn.h): the energy
// program runs in the static scratch of noalloc.cu.  Nothing here calls
// cudaMalloc/cudaFree or copies memory: the leaf descriptors travel as
// kernel parameters, so the call only queues kernel launches.
tn_status tn_energy_noalloc(tn_ctx *ctx, const float *J_dev, const float *h_dev, float *E_dev,
                            void *cuda_stream) {
  Nvtx nv("tn_energy_noalloc");
  if (!ctx) return TN_EINVAL;
  if (ctx->e_scale != 1.0) return fail(ctx, TN_ESTATE, "Max-2-SAT contexts have no noalloc path");
  if (!E_dev) return fail(ctx, TN_EINVAL, "E_dev is NULL");
  if (ctx->net.m > 0 && !J_dev) return fail(ctx, TN_EINVAL, "J_dev is NULL");
  if (!ctx->net.h.empty() && !h_dev)
    return fail(ctx, TN_EINVAL, "the instance has fields: h_dev is required");
  if (!ctx->ordered) return fail(ctx, TN_ESTATE, "tn_order has not been called");
  uint64_t fp = 1469598103934665603ull;
  for (auto &st : ctx->plan.steps) {
    fp = (fp ^ (uint64_t)(st.a + 7)) * 1099511628211ull;
    fp = (fp ^ (uint64_t)(st.b + 7)) * 1099511628211ull;
    fp = (fp ^ (uint64_t)(st.c + 7)) * 1099511628211ull;
  }
  if (!ctx->prog_noalloc || ctx->noalloc_fp != fp) {
    std::unique_ptr<Program> pg(new Program());
    std::string err;
    if (!build_program(ctx->net, ctx->plan, PM_ENERGY, ctx->dt, 0, 0, pg.get(), &err))
      return fail(ctx, TN_EINVAL, err);
    ctx->prog_noalloc = std::move(pg);
    ctx->noalloc_fp = fp;
  }
  Program &p = *ctx->prog_noalloc;
  const int64_t need = p.arena_bytes;
  const int64_t cap = (int64_t)noalloc_scratch_bytes();
  if (need > cap)
    return fail(ctx, TN_ENOMEM, "tn_energy_noalloc: this plan needs " + std::to_string(need) +
                                    " bytes of scratch; the static scratch holds " +
                                    std::to_string(cap) + " bytes (use tn_energy)");
  char *base = nullptr;
  CK(noalloc_scratch(&base));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  PrimeSet ps;
  for (int i = 0; i < TN_MAX_PRIMES; ++i) ps.c[i] = kPrimeC[i];
  ps.r32 = 0;
  auto X = [&](const Loc &l) -> void * { return l.buf < 0 ? nullptr : base + abs_off(p, l); };
  const Batch one;
  // this call only queues work: no GEMM tile timing (it would wait on the stream)
  struct NoTune {
    bool was;
    NoTune() : was(set_gemm_autotune(false)) {}
    ~NoTune() { set_gemm_autotune(was); }
  } no_tune;
  for (const Op &op : p.ops) {
    cudaError_t e = cudaSuccess;
    switch (op.kind) {
      case OP_LEAVES:
        e = launch_leaves_param(p.dt, p.q, p.leaves.data(), (int)p.leaves.size(), J_dev, h_dev,
                                base, st);
        break;
      case OP_PERM:
        e = launch_permute(p.perms[op.idx], X(op.in0), X(op.out), nullptr, nullptr, one, st);
        break;
      case OP_GATE:
        e = launch_gate(p.dt, p.gates[op.idx], X(op.in0), X(op.in1), X(op.out), nullptr,
                        nullptr, nullptr, ps, one, st);
        break;
      case OP_GEMM:
        e = launch_mpgemm(p.dt, p.gemms[op.idx], X(op.in0), X(op.in1), X(op.out), one, st);
        break;
      case OP_TRACE:
        break;
      case OP_CHAIN:
        e = launch_chain(p.dt, p.chains[op.idx], base, X(op.in0), nullptr, X(op.out), nullptr, ps,
                         one, st);
        break;
    }
    if (e != cudaSuccess)
      return fail(ctx, TN_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  }
  CK(launch_energy_out(p.dt, X(p.root), E_dev, st));
  return TN_OK;
}

tn_status tn_maxplus_gemm(int32_t dtype, int64_t batch, int64_t M, int64_t N, int64_t K,
                          const void *A, int32_t transA, const void *B, int32_t transB, void *C,
                          void *cuda_stream) {
  if ((dtype != TN_DTYPE_F32 && dtype != TN_DTYPE_I32) || batch < 0 || M < 0 || N < 0 || K < 1)
    return fail(nullptr, TN_EINVAL, "tn_maxplus_gemm: bad dtype or sizes");
  if (batch * M * N == 0) return TN_OK;
  if (!A || !B || !C) return fail(nullptr, TN_EINVAL, "tn_maxplus_gemm: NULL operand");
  GemmParams g{};
  g.batch = batch;
  g.M = M;
  g.N = N;
  g.K = K;
  g.sAb = M * K;
  g.sAm = transA ? 1 : K;
  g.sAk = transA ? M : 1;
  g.sBb = K * N;
  g.sBk = transB ? 1 : N;
  g.sBn = transB ? K : 1;
  g.sCb = M * N;
  g.sCm = N;
  g.sCn = 1;
  Batch one;
  cudaError_t e = launch_mpgemm(dtype == TN_DTYPE_F32 ? DT_F32 : DT_I32, g, A, B, C, one,
                                (cudaStream_t)cuda_stream);
  if (e != cudaSuccess)
    return fail(nullptr, TN_ECUDA, std::string("tn_maxplus_gemm: ") + cudaGetErrorString(e));
  return TN_OK;
}

tn_status tn_sample(tn_ctx *ctx, int32_t n_samples, uint64_t seed, const int32_t *order,
                    int8_t *sigma) {
  if (!ctx) return TN_EINVAL;
  if (n_samples < 0 || (n_samples > 0 && !sigma)) return fail(ctx, TN_EINVAL, "bad sample buffer");
  if (!ctx->ordered) return fail(ctx, TN_ESTATE, "tn_order has not run");
  const Net &n = ctx->net;
  if (n.q != 2) return fail(ctx, TN_EINVAL, "sampling is Ising only (q == 2)");
  if (ctx->dt != DT_I32)
    return fail(ctx, TN_EINVAL, "sampling needs integral couplings (an INT32 context)");
  if (!ctx->host_couplings)
    return fail(ctx, TN_ESTATE, "couplings were last set on the device; set them from the host");
  std::vector<int> ord(n.n);
  if (order) {
    std::vector<char> seen(n.n, 0);
    for (int i = 0; i < n.n; ++i) {
      const int v = order[i];
      if (v < 0 || v >= n.n || seen[v]) return fail(ctx, TN_EINVAL, "order is not a permutation");
      seen[v] = 1;
      ord[i] = v;
    }
  } else {
    for (int i = 0; i < n.n; ++i) ord[i] = i;
  }
  // pinned instances: |values| stay below the INT32 sentinel margin
  double mag = n.n + 1.0;
  for (float x : n.J) mag += std::fabs(x);
  for (float x : n.h) mag += std::fabs(x);
  if (mag >= (double)(1 << 29)) return fail(ctx, TN_EINVAL, "couplings too large to pin exactly");
  // the same graph and plan, with fields on every spin (zeros if it has none)
  std::vector<int32_t> e(2 * (size_t)std::max(n.m, 1));
  for (int k = 0; k < n.m; ++k) {
    e[2 * k] = n.eu[k];
    e[2 * k + 1] = n.ev[k];
  }
  std::vector<float> h0 = n.h.empty() ? std::vector<float>(n.n, 0.f) : n.h;
  tn_ctx *pc = nullptr;
  tn_status s = tn_build(&pc, n.n, n.m, e.data(), n.J.data(), h0.data(), 2, TN_DTYPE_I32);
  if (s != TN_OK) return fail(ctx, s, "sampler: " + g_build_err);
  std::unique_ptr<tn_ctx, void (*)(tn_ctx *)> guard(pc, tn_destroy);
  pc->plan = ctx->plan;
  pc->ordered = true;
  pc->stream = ctx->stream;
  std::vector<float> Jrep;
  CountFn fn = [&](const std::vector<float> &h, int K, std::vector<double> *E,
                   std::vector<Big> *cnt) -> int {
    Jrep.assign((size_t)std::max(1, K * n.m), 0.f);
    for (int k = 0; k < K; ++k) std::copy(n.J.begin(), n.J.end(), Jrep.begin() + (size_t)k * n.m);
    std::vector<uint64_t> limbs((size_t)K * 3);
    std::vector<int32_t> st(K, 0);
    E->assign(K, 0.0);
    tn_status r = tn_count_batch(pc, K, Jrep.data(), h.data(), 0, 3, limbs.data(), 3, E->data(),
                                 st.data());
    if (r != TN_OK) {
      fail(ctx, r, "sampler: " + pc->err);
      return (int)r;
    }
    cnt->assign(K, Big());
    for (int k = 0; k < K; ++k) (*cnt)[k].assign(limbs.begin() + 3 * k, limbs.begin() + 3 * k + 3);
    return 0;
  };
  std::vector<int8_t> out;
  std::string err;
  const int rc = sample_ground_states(n.n, n_samples, ord, h0, seed, 16, fn, &out, &err);
  if (rc == -1) return fail(ctx, TN_ESTATE, err);
  if (rc) return (tn_status)rc;
  std::copy(out.begin(), out.end(), sigma);
  return TN_OK;
}

const char *tn_last_error(const tn_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_build_err.c_str();
}

void tn_destroy(tn_ctx *ctx) {
  if (!ctx) return;
  for (auto &p : ctx->prog) if (p) free_program(p.get());
  if (ctx->prog_pass) free_program(ctx->prog_pass.get());
  if (ctx->dev_ready) {
    cudaFree(ctx->d_J);
    cudaFree(ctx->d_h);
    cudaFree(ctx->d_eu);
    cudaFree(ctx->d_ev);
    cudaFree(ctx->d_state);
    cudaFree(ctx->d_out);
    cudaFree(ctx->d_err);
  }
  if (ctx->d_Jb) cudaFree(ctx->d_Jb);
  if (ctx->d_hb) cudaFree(ctx->d_hb);
  if (ctx->d_stateb) cudaFree(ctx->d_stateb);
  if (ctx->d_outb) cudaFree(ctx->d_outb);
  if (ctx->d_arena) cudaFree(ctx->d_arena);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

}  // extern "C"
