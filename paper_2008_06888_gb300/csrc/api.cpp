// api.cpp -- the C ABI of include/tn.h: contexts, execution of the lowered
// programs on the device, and exact count reconstruction (CRT).
#include "../../include/tn.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "kernels.h"
#include "planner.h"
#include "program.h"

using namespace tn;

// 61-bit primes p_i = 2^61 - c_i; the last one used by a call is the witness.
static const uint64_t kPrimeC[TN_MAX_PRIMES] = {1, 31, 45, 229, 259, 283, 339, 391, 403};

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
  int prog_P = 0;
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
  // host-side program of tn_energy_noalloc and the plan fingerprint it was built for
  std::unique_ptr<Program> prog_noalloc;
  uint64_t noalloc_fp = 0;
};

static std::string g_build_err;

namespace {

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

tn_status get_program(tn_ctx *ctx, ProgMode mode, int P, Program **out) {
  if (!ctx->ordered) return fail(ctx, TN_ESTATE, "tn_order has not been called");
  std::unique_ptr<Program> &slot = ctx->prog[mode];
  if (!slot || (mode == PM_COUNT && ctx->prog_P != P)) {
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
                       slot.get(), &err)) {
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
    if (mode == PM_COUNT) ctx->prog_P = P;
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

tn_status run_ops(tn_ctx *ctx, Program &p, int op_begin, int op_end, cudaStream_t st,
                  bool account) {
  char *ar = ctx->d_arena;
  PrimeSet ps;
  for (int i = 0; i < TN_MAX_PRIMES; ++i) ps.c[i] = kPrimeC[i];
  auto X = [&](const Loc &l) -> void * { return l.buf < 0 ? nullptr : ar + abs_off(p, l); };
  auto Nn = [&](const Loc &l) -> uint64_t * {
    return l.buf < 0 ? nullptr : (uint64_t *)(ar + p.bufs[l.buf].off + l.noff);
  };
  if (p.mode == PM_CONFIG && op_end > p.fwd_end)
    CK(cudaMemsetAsync(ctx->d_state, 0xff, std::max(1, ctx->net.n), st));
  if (ctx->profiling && ctx->ev_next > 4096) collect_profile(ctx);
  for (int oi = op_begin; oi < op_end; ++oi) {
    const Op &op = p.ops[oi];
    cudaError_t e = cudaSuccess;
    const int slot = op_kind_slot(op.kind);
    int e0 = -1;
    if (ctx->profiling) {
      e0 = ctx->ev_next;
      cudaEventRecord(next_event(ctx), st);
    }
    switch (op.kind) {
      case OP_LEAVES:
        e = launch_leaves(p.dt, p.q, p.d_leaves, (int)p.leaves.size(), ctx->d_J, ctx->d_h, ar, p.P,
                          st);
        break;
      case OP_PERM:
        e = launch_permute(p.perms[op.idx], X(op.in0), X(op.out), Nn(op.in0), Nn(op.out), st);
        break;
      case OP_GATE:
        e = launch_gate(p.dt, p.gates[op.idx], X(op.in0), X(op.in1), X(op.out), Nn(op.in0),
                        Nn(op.in1), Nn(op.out), ps, st);
        break;
      case OP_GEMM:
        e = launch_gemm(p.dt, p.gemms[op.idx], X(op.in0), X(op.in1), X(op.out), st);
        if (e == cudaSuccess && p.P > 0)
          e = launch_gemm_count(p.dt, p.gemms[op.idx], X(op.in0), X(op.in1), X(op.out),
                                Nn(op.in0), Nn(op.in1), Nn(op.out), ps, st);
        break;
      case OP_TRACE:
        e = launch_trace(p.dt, p.q, p.d_trace + op.trace_begin, op.trace_n, p.d_chain_traces,
                         p.trace_smem, ar, ctx->d_state, ctx->net.n, ctx->d_err, st);
        break;
      case OP_CHAIN:
        e = launch_chain(p.dt, p.chains[op.idx], ar, X(op.in0), Nn(op.in0), X(op.out), Nn(op.out),
                         ps, st);
        break;
    }
    if (e != cudaSuccess)
      return fail(ctx, TN_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    int nl = 1;
    if (op.kind == OP_GEMM && p.P > 0) nl = 2;
    if (op.kind == OP_PERM && p.P > 0) nl = 2;
    if (account) {
      ctx->launches[slot] += nl;
      ctx->prof_bytes[slot] += op.bytes;
      ctx->prof_macs[slot] += op.macs;
    }
    if (ctx->profiling) {
      int e1 = ctx->ev_next;
      cudaEventRecord(next_event(ctx), st);
      ctx->pending.push_back({slot, e0, e1});
    }
  }
  return TN_OK;
}

void account_range(tn_ctx *ctx, const Program &p, int b, int e) {
  for (int oi = b; oi < e; ++oi) {
    const Op &op = p.ops[oi];
    const int slot = op_kind_slot(op.kind);
    int nl = 1;
    if ((op.kind == OP_GEMM || op.kind == OP_PERM) && p.P > 0) nl = 2;
    ctx->launches[slot] += nl;
    ctx->prof_bytes[slot] += op.bytes;
    ctx->prof_macs[slot] += op.macs;
  }
}

// Eager on the first run of a range (and whenever profiling, or with
// TN_NO_GRAPH set); captured into a CUDA graph on the second run and
// replayed from then on.
tn_status run_program(tn_ctx *ctx, Program &p, int op_begin = 0, int op_end = -1) {
  if (op_end < 0) op_end = (int)p.ops.size();
  static const bool no_graph = std::getenv("TN_NO_GRAPH") != nullptr;
  if (ctx->profiling || no_graph) return run_ops(ctx, p, op_begin, op_end, ctx->stream, true);
  Program::Graph *g = nullptr;
  for (auto &x : p.graphs)
    if (x.begin == op_begin && x.end == op_end) g = &x;
  if (g && g->arena != ctx->d_arena) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    g->runs = 0;
    g->arena = ctx->d_arena;
  }
  if (!g) {
    p.graphs.push_back(Program::Graph{op_begin, op_end, 0, ctx->d_arena, nullptr});
    g = &p.graphs.back();
  }
  if (!g->exec && g->runs == 0) {
    g->runs = 1;
    return run_ops(ctx, p, op_begin, op_end, ctx->stream, true);
  }
  if (!g->exec) {
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    tn_status s = run_ops(ctx, p, op_begin, op_end, ctx->cap_stream, false);
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
  account_range(ctx, p, op_begin, op_end);
  return TN_OK;
}

double root_energy(const tn_ctx *ctx, const void *raw) {
  if (ctx->dt == DT_F32) {
    float v;
    std::memcpy(&v, raw, 4);
    return -(double)v;
  }
  int32_t v;
  std::memcpy(&v, raw, 4);
  return -(double)v;
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
    ok = tree_greedy(ctx->net, seed, restarts, cm, &t, &err);
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
    return TN_OK;
  }
  tn_status s = ensure_device(ctx);
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
    CK(launch_state_out(ctx->net.q, ctx->net.n, ctx->d_state, ctx->d_out, ctx->stream));
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
  if (!ctx->have_state) return fail(ctx, TN_ESTATE, "tn_config has not run");
  const Net &n = ctx->net;
  if (on_device) {
    CK(launch_grad(n.q, n.n, n.m, ctx->d_eu, ctx->d_ev, ctx->d_state, dJ, dh, ctx->stream));
    return TN_OK;
  }
  float *gJ = nullptr, *gh = nullptr;
  CK(cudaMalloc(&gJ, std::max(1, n.m) * sizeof(float)));
  CK(cudaMalloc(&gh, std::max(1, n.n) * sizeof(float)));
  CK(launch_grad(n.q, n.n, n.m, ctx->d_eu, ctx->d_ev, ctx->d_state, gJ, gh, ctx->stream));
  if (dJ && n.m) CK(cudaMemcpyAsync(dJ, gJ, n.m * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (dh) CK(cudaMemcpyAsync(dh, gh, n.n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  cudaFree(gJ);
  cudaFree(gh);
  return TN_OK;
}

tn_status tn_count(tn_ctx *ctx, int32_t n_primes, uint64_t *limbs, int32_t *n_limbs,
                   double *ln_count, double *E) {
  if (!ctx) return TN_EINVAL;
  ctx->fwd_done = false;
  if (n_primes < 1 || n_primes > TN_MAX_PRIMES - 1)
    return fail(ctx, TN_EINVAL, "n_primes must be in [1, 8]");
  tn_status s = ensure_device(ctx);
  if (s != TN_OK) return s;
  const int P = n_primes + 1;  // + witness
  Program *p;
  if ((s = get_program(ctx, PM_COUNT, P, &p)) != TN_OK) return s;
  if ((s = run_program(ctx, *p)) != TN_OK) return s;
  char raw[4];
  std::vector<uint64_t> res(P);
  const char *base = ctx->d_arena + p->bufs[p->root.buf].off;
  CK(cudaMemcpyAsync(raw, base + p->root.xoff, 4, cudaMemcpyDeviceToHost, ctx->stream));
  for (int i = 0; i < P; ++i)
    CK(cudaMemcpyAsync(&res[i], base + p->root.noff + (int64_t)i * p->root.plane * 8, 8,
                       cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (E) *E = root_energy(ctx, raw);
  std::vector<uint64_t> r(res.begin(), res.begin() + n_primes), pr;
  for (int i = 0; i < n_primes; ++i) pr.push_back((1ull << 61) - kPrimeC[i]);
  std::vector<uint64_t> v = crt(r, pr);
  uint64_t pw = (1ull << 61) - kPrimeC[n_primes];
  if (limbs_mod(v, pw) != res[n_primes])
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

tn_status tn_batch_run(int32_t B, tn_ctx *const *ctxs, double *E, uint64_t *limbs,
                       int32_t limbs_per, int32_t *status) {
  tn_status first = TN_OK;
  for (int k = 0; k < B; ++k) {
    tn_ctx *c = ctxs[k];
    tn_status s;
    if (limbs) {
      int32_t nl = limbs_per;
      s = tn_count(c, 3, limbs + (int64_t)k * limbs_per, &nl, nullptr, E ? &E[k] : nullptr);
    } else {
      s = E ? tn_energy(c, &E[k]) : TN_EINVAL;
    }
    if (status) status[k] = s;
    if (s != TN_OK && first == TN_OK) first = s;
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
    if (!build_program(ctx->net, ctx->plan, PM_COUNT, ctx->dt, 4, 0, &pn, &err)) return TN_EINVAL;
    *arena_count = pn.arena_bytes;
  }
  return TN_OK;
}

// For callers that cannot allocate device memory (see tn.h): the energy
// program runs in the static scratch of noalloc.cu.  Nothing here calls
// cudaMalloc/cudaFree; the only device traffic besides the kernels is one
// host-to-device copy of the leaf descriptors into the scratch.
tn_status tn_energy_noalloc(tn_ctx *ctx, const float *J_dev, const float *h_dev, float *E_dev,
                            void *cuda_stream) {
  if (!ctx) return TN_EINVAL;
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
  const int64_t leaves_off = (p.arena_bytes + 255) / 256 * 256;
  const int64_t need = leaves_off + (int64_t)(p.leaves.size() * sizeof(LeafDesc));
  const int64_t cap = (int64_t)noalloc_scratch_bytes();
  if (need > cap)
    return fail(ctx, TN_ENOMEM, "tn_energy_noalloc: this plan needs " + std::to_string(need) +
                                    " bytes of scratch; the static scratch holds " +
                                    std::to_string(cap) + " bytes (use tn_energy)");
  char *base = nullptr;
  CK(noalloc_scratch(&base));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  LeafDesc *d_leaves = reinterpret_cast<LeafDesc *>(base + leaves_off);
  if (!p.leaves.empty())
    CK(cudaMemcpyAsync(d_leaves, p.leaves.data(), p.leaves.size() * sizeof(LeafDesc),
                       cudaMemcpyHostToDevice, st));
  PrimeSet ps;
  for (int i = 0; i < TN_MAX_PRIMES; ++i) ps.c[i] = kPrimeC[i];
  auto X = [&](const Loc &l) -> void * { return l.buf < 0 ? nullptr : base + abs_off(p, l); };
  for (const Op &op : p.ops) {
    cudaError_t e = cudaSuccess;
    switch (op.kind) {
      case OP_LEAVES:
        e = launch_leaves(p.dt, p.q, d_leaves, (int)p.leaves.size(), J_dev, h_dev, base, 0, st);
        break;
      case OP_PERM:
        e = launch_permute(p.perms[op.idx], X(op.in0), X(op.out), nullptr, nullptr, st);
        break;
      case OP_GATE:
        e = launch_gate(p.dt, p.gates[op.idx], X(op.in0), X(op.in1), X(op.out), nullptr,
                        nullptr, nullptr, ps, st);
        break;
      case OP_GEMM:
        e = launch_gemm(p.dt, p.gemms[op.idx], X(op.in0), X(op.in1), X(op.out), st);
        break;
      case OP_TRACE:
        break;
      case OP_CHAIN:
        e = launch_chain(p.dt, p.chains[op.idx], base, X(op.in0), nullptr, X(op.out), nullptr, ps,
                         st);
        break;
    }
    if (e != cudaSuccess)
      return fail(ctx, TN_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  }
  CK(launch_energy_out(p.dt, X(p.root), E_dev, st));
  return TN_OK;
}

const char *tn_last_error(const tn_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_build_err.c_str();
}

void tn_destroy(tn_ctx *ctx) {
  if (!ctx) return;
  for (auto &p : ctx->prog) if (p) free_program(p.get());
  if (ctx->dev_ready) {
    cudaFree(ctx->d_J);
    cudaFree(ctx->d_h);
    cudaFree(ctx->d_eu);
    cudaFree(ctx->d_ev);
    cudaFree(ctx->d_state);
    cudaFree(ctx->d_out);
    cudaFree(ctx->d_err);
  }
  if (ctx->d_arena) cudaFree(ctx->d_arena);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

}  // extern "C"
