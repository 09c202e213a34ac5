// program.cpp -- lowering of classified steps to kernel launches, static
// arena planning, and the checkpoint / recompute schedule of the traceback.
//
// Each pairwise step C = A (.) B (Sec. III) becomes either
//   * a gate contraction when one operand contributes few states (K and N
//     small): the big operand is read in place through per-leg strides, so no
//     transpose is needed; this covers the sweep steps of a lattice, the
//     Hadamard-type steps with K = 1 and the unary reductions; or
//   * a strided batched max-plus GEMM over [batch][M][K] x [batch][K][N],
//     preceded by a transpose of any operand whose legs of one class are not
//     contiguous in memory.
#include "program.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>

namespace tn {

namespace {

constexpr int64_t kAlign = 256;
inline int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int64_t ipow(int q, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= q;
  return r;
}

int pos_of(const std::vector<int> &v, int x) {
  for (int i = 0; i < (int)v.size(); ++i) if (v[i] == x) return i;
  return -1;
}

// ---- folding a register chain's diagonal gates into its replace gates.
//
// A diagonal term D that does not depend on the digit a replace gate
// eliminates commutes with that gate's max, and one that depends on the
// digit the gate creates can be added after it: so D is added into the
// table of the replace gate that last created one of D's register legs
// ("post"), else of the first one that later eliminates one of them ("pre"),
// provided D's other legs keep their spins in between.  Terms on fixed legs
// only are per-thread constants and go into any replace gate.  Diagonal
// gates that fit nowhere remain table gates of their own.  A final
// contraction (a replace gate without a new digit) takes terms like the
// replace gate that next eliminates their leg.

static bool tg_fixed_bit(TGate &t, int sh, int8_t *bit) {
  for (int i = 0; i < t.nf; ++i)
    if (t.fsh[i] == sh) { *bit = (int8_t)(3 + i); return true; }
  if (t.nf >= TN_TG_MAXF) return false;
  t.fsh[t.nf] = (int8_t)sh;
  *bit = (int8_t)(3 + t.nf);
  t.nf++;
  return true;
}

// add diagonal gate d of cp into replace table t; jbit: table bit of the leg
// on t's register bit J (0 pre, 1 post)
static bool tg_add_diag(const ChainParams &cp, int d, TGate &t, int jbit) {
  if (t.ncomp >= TN_TG_MAXC) return false;
  TGate u = t;
  const ChainGate &g = cp.g[d];
  const int c = u.ncomp;
  u.cg[c] = (int8_t)d;
  u.cbit[c][0] = u.cbit[c][1] = u.cbit[c][2] = u.cbit[c][3] = -1;
  for (int l = 0; l < g.nb; ++l) {
    int8_t bit;
    if (g.lsb[l] < 0) {
      if (!tg_fixed_bit(u, g.lrank[l], &bit)) return false;
    } else if (g.lsb[l] == u.J) {
      if (jbit < 0) return false;
      bit = (int8_t)jbit;
    } else {
      if (u.K >= 0 && u.K != g.lsb[l]) return false;
      u.K = (int8_t)g.lsb[l];
      bit = 2;
    }
    u.cbit[c][2 + l] = bit;
  }
  u.ncomp++;
  t = u;
  return true;
}

static void fold_reg_chain(ChainParams &cp) {
  const int n = cp.ngates;
  std::vector<TGate> tg;
  std::vector<int> at;               // position of each table gate in the chain
  std::vector<int> of(n, -1);        // replace gate -> its table gate
  for (int i = 0; i < n; ++i) {
    const ChainGate &g = cp.g[i];
    if (g.kind != 0 && g.kind != 2) continue;
    TGate t{};
    t.kind = (int8_t)g.kind;   // 0 replace, 2 contract (no new digit)
    t.J = (int8_t)g.ls;
    t.K = -1;
    t.kspin = g.kspin;
    t.cg[0] = (int8_t)i;
    t.cbit[0][0] = 0;
    t.cbit[0][1] = g.kind == 0 ? 1 : -1;
    t.cbit[0][2] = t.cbit[0][3] = -1;
    // its own extra legs: a register leg takes the K slot (the builder admits at
    // most one), a fixed leg a fixed slot
    for (int l = 0; l < g.nb; ++l) {
      if (g.lsb[l] >= 0) {
        t.K = (int8_t)g.lsb[l];
        t.cbit[0][2 + l] = 2;
      } else {
        tg_fixed_bit(t, g.lrank[l], &t.cbit[0][2 + l]);
      }
    }
    t.ncomp = 1;
    of[i] = (int)tg.size();
    tg.push_back(t);
    at.push_back(i);
  }
  auto last_rep = [&](int r, int p) {
    for (int i = p - 1; i >= 0; --i)
      if (cp.g[i].kind == 0 && cp.g[i].ls == r) return i;
    return -1;
  };
  for (int d = 0; d < n; ++d) {
    const ChainGate &g = cp.g[d];
    if (g.kind != 1) continue;
    std::vector<int> regs;
    for (int l = 0; l < g.nb; ++l)
      if (g.lsb[l] >= 0) regs.push_back(g.lsb[l]);
    bool done = false;
    if (regs.empty()) {
      for (size_t k = 0; k < tg.size() && !done; ++k) done = tg_add_diag(cp, d, tg[k], -1);
    } else {
      int cs = -1;
      for (int r : regs) cs = std::max(cs, last_rep(r, d));
      if (cs >= 0) done = tg_add_diag(cp, d, tg[of[cs]], 1);
      if (!done) {
        for (int j = d + 1; j < n; ++j) {
          if (cp.g[j].kind != 0 && cp.g[j].kind != 2) continue;
          if (std::find(regs.begin(), regs.end(), cp.g[j].ls) == regs.end()) continue;
          done = tg_add_diag(cp, d, tg[of[j]], 0);
          break;
        }
      }
    }
    if (done) continue;
    TGate t{};
    t.kind = 1;
    t.J = regs.size() > 0 ? (int8_t)regs[0] : (int8_t)-1;
    t.K = regs.size() > 1 ? (int8_t)regs[1] : (int8_t)-1;
    if (t.K >= 0 && t.K < t.J) std::swap(t.J, t.K);
    t.kspin = -1;
    t.cg[0] = (int8_t)d;
    t.cbit[0][0] = t.cbit[0][1] = t.cbit[0][2] = t.cbit[0][3] = -1;
    for (int l = 0; l < g.nb; ++l) {
      int8_t bit = -1;
      if (g.lsb[l] < 0) tg_fixed_bit(t, g.lrank[l], &bit);   // at most 2 of 3 slots
      else bit = g.lsb[l] == t.J ? 0 : 1;
      t.cbit[0][2 + l] = bit;
    }
    t.ncomp = 1;
    tg.push_back(t);
    at.push_back(d);
  }
  std::vector<int> ord(tg.size());
  for (size_t k = 0; k < ord.size(); ++k) ord[k] = (int)k;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return at[a] < at[b]; });
  int off = 0;
  cp.ntg = (int)tg.size();
  for (size_t k = 0; k < ord.size(); ++k) {
    TGate t = tg[ord[k]];
    for (int i = t.nf; i < TN_TG_MAXF; ++i) t.fsh[i] = 62;   // a tau bit that is always 0
    // dispatch code: replace J * 7 + K + 1 (< 42), diagonal 42 + (J + 1) * 7 + K + 1,
    // contract 100 + J * 7 + K + 1 (always the last table gate)
    t.code = t.kind == 0   ? (int16_t)(t.J * 7 + (t.K + 1))
             : t.kind == 2 ? (int16_t)(100 + t.J * 7 + (t.K + 1))
                           : (int16_t)(42 + (t.J + 1) * 7 + (t.K + 1));
    t.toff = (int16_t)off;
    off += 8 << t.nf;
    cp.tg[k] = t;
  }
  cp.ttotal = off;
}

struct Builder {
  const Net &net;
  const Plan &plan;
  Program &pr;
  int q, P;
  int rb;                                // bytes of one residue
  std::vector<std::vector<int>> order;   // memory leg order of each plan tensor
  std::vector<Loc> loc;
  std::string err;

  // unit[t]: every count of tensor t is 1 (leaves, and steps that contract
  // nothing from unit inputs: outer products and Hadamard-type steps)
  std::vector<char> unit;

  Builder(const Net &n, const Plan &p, Program &r)
      : net(n), plan(p), pr(r), q(r.q), P(r.P), rb(r.rbytes), order(p.legset.size()),
        loc(p.legset.size()),
        unit(p.legset.size(), 0) {
    for (int i = 0; i < p.n_leaves; ++i) unit[i] = 1;
    for (const PStep &st : p.steps)
      unit[st.c] = unit[st.a] && (st.b < 0 || unit[st.b]) && st.K.empty();
  }

  int64_t stride(const std::vector<int> &ord, int leg) const {
    int p = pos_of(ord, leg);
    if (p < 0) return 0;
    return ipow(q, (int)ord.size() - 1 - p);
  }

  Loc new_tensor(int64_t elems) {
    BufInfo b;
    int64_t xb = align_up(elems * 4);
    b.bytes = xb + (P > 0 ? align_up((int64_t)P * elems * rb) : 0);
    if (b.bytes == 0) b.bytes = kAlign;
    pr.bufs.push_back(b);
    Loc l;
    l.buf = (int)pr.bufs.size() - 1;
    l.xoff = 0;
    l.noff = xb;
    l.plane = elems;
    return l;
  }
  void use(const Loc &l, int op) {
    if (l.buf < 0) return;
    BufInfo &b = pr.bufs[l.buf];
    b.first = std::min(b.first, op);
    b.last = std::max(b.last, op);
  }
  double elem_bytes() const { return 4.0 + (double)rb * P; }
  int push(Op op) {
    auto el = [&](const Loc &l) { return l.buf < 0 ? 0.0 : (double)l.plane; };
    if (op.kind == OP_PERM) op.bytes = 2 * el(op.out) * elem_bytes();
    else if (op.kind == OP_LEAVES) op.bytes = el(op.out) * elem_bytes();
    else op.bytes = (el(op.in0) + el(op.in1) + el(op.out)) * elem_bytes();
    pr.ops.push_back(op);
    int i = (int)pr.ops.size() - 1;
    use(op.in0, i);
    use(op.in1, i);
    use(op.out, i);
    return i;
  }

  // ---- leaves
  void emit_leaves() {
    int64_t total = 0;
    for (int i = 0; i < plan.n_leaves; ++i) {
      pr.leaf_elem.push_back(total);
      total += ipow(q, (int)plan.legset[i].size());
    }
    Loc L = new_tensor(total);
    pr.leaves_loc = L;
    for (int i = 0; i < plan.n_leaves; ++i) {
      order[i] = plan.legset[i];
      Loc l = L;
      l.xoff = L.xoff + pr.leaf_elem[i] * 4;
      l.noff = L.noff + pr.leaf_elem[i] * rb;
      loc[i] = l;
    }
    Op op;
    op.kind = OP_LEAVES;
    op.out = L;
    push(op);
  }

  // ---- permutation of tensor t into `to` (new buffer); returns its location
  Loc emit_perm(int t, const std::vector<int> &to) {
    const std::vector<int> &from = order[t];
    PermParams pp{};
    std::vector<int64_t> dims, sin;
    for (int l : to) {
      dims.push_back(q);
      sin.push_back(stride(from, l));
    }
    // merge runs of output legs that are adjacent in the input too
    std::vector<int64_t> md, ms;
    for (size_t j = 0; j < dims.size(); ++j) {
      if (!md.empty() && ms.back() == sin[j] * dims[j]) {
        md.back() *= dims[j];
        ms.back() = sin[j];
      } else {
        md.push_back(dims[j]);
        ms.push_back(sin[j]);
      }
    }
    pp.r = (int)md.size();
    pp.total = ipow(q, (int)to.size());
    for (int j = 0; j < pp.r; ++j) { pp.dims[j] = md[j]; pp.sin[j] = ms[j]; }
    Loc out = new_tensor(pp.total);
    pp.planeIn = loc[t].plane;
    pp.planeOut = out.plane;
    pp.P = P;
    pp.rbytes = rb;
    pr.perms.push_back(pp);
    Op op;
    op.kind = OP_PERM;
    op.in0 = loc[t];
    op.out = out;
    op.idx = (int)pr.perms.size() - 1;
    push(op);
    pr.n_transposes++;
    return out;
  }

  // ---- gate contraction: A big (in place), B small or absent.
  // K and N legs are given in the order that defines k and n.
  bool make_gate(const std::vector<int> &ordA, const std::vector<int> *ordB,
                 const std::vector<int> &K, const std::vector<int> &N, GateParams *g,
                 std::vector<int> *ordC) {
    GateParams &p = *g;
    p = GateParams{};
    std::vector<int> outer;
    for (int l : ordA) if (pos_of(K, l) < 0) outer.push_back(l);
    *ordC = outer;
    ordC->insert(ordC->end(), N.begin(), N.end());
    int64_t Ks = ipow(q, (int)K.size()), Ns = ipow(q, (int)N.size());
    if (Ks > TN_GATE_MAX_K || Ns > TN_GATE_MAX_N) return false;
    // segments, innermost first, then reversed
    std::vector<int64_t> sz, sa, sb, sc;
    for (int j = (int)outer.size() - 1; j >= 0; --j) {
      int l = outer[j];
      int64_t a = stride(ordA, l), b = ordB ? stride(*ordB, l) : 0, c = stride(*ordC, l);
      if (!sz.empty() && a == sa.back() * sz.back() && b == sb.back() * sz.back() &&
          c == sc.back() * sz.back()) {
        sz.back() *= q;
      } else {
        sz.push_back(q);
        sa.push_back(a);
        sb.push_back(b);
        sc.push_back(c);
      }
    }
    if ((int)sz.size() > TN_MAX_SEG) return false;
    p.nseg = (int)sz.size();
    for (int s = 0; s < p.nseg; ++s) {
      int r = p.nseg - 1 - s;
      p.seg_size[s] = sz[r];
      p.seg_sA[s] = sa[r];
      p.seg_sB[s] = sb[r];
      p.seg_sC[s] = sc[r];
      p.seg_sh[s] = -1;
      for (int b = 0; b < 62; ++b)
        if ((int64_t(1) << b) == sz[r]) p.seg_sh[s] = b;
    }
    p.outer = ipow(q, (int)outer.size());
    p.Ks = (int)Ks;
    p.Ns = (int)Ns;
    p.hasB = ordB ? 1 : 0;
    for (int64_t k = 0; k < Ks; ++k) {
      int64_t r = k, oa = 0, ob = 0;
      for (int j = (int)K.size() - 1; j >= 0; --j) {
        int64_t d = r % q;
        r /= q;
        oa += d * stride(ordA, K[j]);
        if (ordB) ob += d * stride(*ordB, K[j]);
      }
      p.kA[k] = oa;
      p.kB[k] = ob;
    }
    for (int64_t n = 0; n < Ns; ++n) {
      int64_t r = n, ob = 0;
      for (int j = (int)N.size() - 1; j >= 0; --j) {
        int64_t d = r % q;
        r /= q;
        if (ordB) ob += d * stride(*ordB, N[j]);
      }
      p.nB[n] = ob;
      p.nC[n] = n;
    }
    p.P = P;
    return true;
  }

  void push_gate(const GateParams &g, const Loc &A, const Loc *B, const Loc &C, bool unitB) {
    GateParams p = g;
    p.unitB = unitB ? 1 : 0;
    p.planeA = A.plane;
    p.planeB = B ? B->plane : 0;
    p.planeC = C.plane;
    pr.gates.push_back(p);
    Op op;
    op.macs = (double)p.outer * p.Ks * p.Ns;
    op.kind = OP_GATE;
    op.in0 = A;
    if (B) op.in1 = *B;
    op.out = C;
    op.idx = (int)pr.gates.size() - 1;
    push(op);
    pr.n_gate++;
  }

  // K legs ordered as in A's memory order
  std::vector<int> k_order(const std::vector<int> &ordA, const std::vector<int> &K) {
    std::vector<int> r;
    for (int l : ordA) if (pos_of(K, l) >= 0) r.push_back(l);
    return r;
  }

  bool emit_unary(const PStep &st) {
    int a = st.a;
    std::vector<int> Krem = k_order(order[a], st.K);
    std::vector<int> cur_ord = order[a];
    Loc cur = loc[a];
    int maxk = 0;
    while (ipow(q, maxk + 1) <= TN_GATE_MAX_K) ++maxk;
    do {
      std::vector<int> chunk(Krem.begin(), Krem.begin() + std::min<size_t>(maxk, Krem.size()));
      Krem.erase(Krem.begin(), Krem.begin() + chunk.size());
      GateParams g;
      std::vector<int> ordC;
      if (!make_gate(cur_ord, nullptr, chunk, {}, &g, &ordC)) {
        // too many segments: canonicalise A first
        int tmp = a;
        (void)tmp;
        err = "unary reduction: layout too fragmented";
        return false;
      }
      Loc out = new_tensor(ipow(q, (int)ordC.size()));
      push_gate(g, cur, nullptr, out, true);
      cur = out;
      cur_ord = ordC;
    } while (!Krem.empty());
    order[st.c] = cur_ord;
    loc[st.c] = cur;
    pr.macs += (double)ipow(q, (int)(st.M.size() + st.K.size()));
    return true;
  }

  // class view of a tensor for the GEMM path: each class contiguous, the
  // innermost leg not a batch leg; returns the class-internal orders.
  bool gemm_view(const std::vector<int> &ord, const std::vector<int> &c0,
                 const std::vector<int> &c1, const std::vector<int> &c2,
                 std::vector<int> *o0, std::vector<int> *o1, std::vector<int> *o2) {
    std::vector<int> cls(ord.size());
    for (size_t i = 0; i < ord.size(); ++i) {
      if (pos_of(c0, ord[i]) >= 0) cls[i] = 0;
      else if (pos_of(c1, ord[i]) >= 0) cls[i] = 1;
      else cls[i] = 2;
    }
    int seen[3] = {0, 0, 0};
    for (size_t i = 0; i < ord.size(); ++i) {
      if (i > 0 && cls[i] != cls[i - 1] && seen[cls[i]]) return false;
      seen[cls[i]] = 1;
    }
    if (!ord.empty() && cls.back() == 0 && (c1.size() + c2.size()) > 0) return false;
    o0->clear(); o1->clear(); o2->clear();
    for (size_t i = 0; i < ord.size(); ++i)
      (cls[i] == 0 ? o0 : cls[i] == 1 ? o1 : o2)->push_back(ord[i]);
    return true;
  }

  int64_t inner_stride(const std::vector<int> &ord, const std::vector<int> &cls) {
    if (cls.empty()) return 0;
    return stride(ord, cls.back());
  }

  struct GemmChoice {
    int A, B;
    std::vector<int> bo, mo, ko, no;   // class orders
    bool permA, permB;
    int64_t cost;
  };

  GemmChoice plan_gemm(int A, int B, const std::vector<int> &batch, const std::vector<int> &M,
                       const std::vector<int> &K, const std::vector<int> &N) {
    GemmChoice ch;
    ch.A = A;
    ch.B = B;
    ch.cost = 0;
    std::vector<int> b0, m0, k0;
    if (gemm_view(order[A], batch, M, K, &b0, &m0, &k0)) {
      ch.permA = false;
    } else {
      ch.permA = true;
      b0.clear(); m0.clear(); k0.clear();
      for (int l : order[A]) {
        if (pos_of(batch, l) >= 0) b0.push_back(l);
        else if (pos_of(M, l) >= 0) m0.push_back(l);
        else k0.push_back(l);
      }
      ch.cost += ipow(q, (int)order[A].size());
    }
    std::vector<int> b1, k1, n1;
    bool okB = gemm_view(order[B], batch, K, N, &b1, &k1, &n1) && b1 == b0 && k1 == k0;
    if (!okB) {
      n1.clear();
      for (int l : order[B]) if (pos_of(N, l) >= 0) n1.push_back(l);
      ch.cost += ipow(q, (int)order[B].size());
    }
    ch.permB = !okB;
    ch.bo = b0; ch.mo = m0; ch.ko = k0; ch.no = n1;
    return ch;
  }

  void emit_pair(const PStep &st) {
    const int a = st.a, b = st.b;
    const int64_t Sa = ipow(q, (int)order[a].size()), Sb = ipow(q, (int)order[b].size());
    const int64_t Sk = ipow(q, (int)st.K.size());
    const int64_t Sm = ipow(q, (int)st.M.size()), Sn = ipow(q, (int)st.N.size());
    pr.macs += (double)ipow(q, (int)(st.batch.size() + st.M.size() + st.N.size() + st.K.size()));
    // gate options: (big, small, new legs of small)
    struct GOpt { int A, B; const std::vector<int> *N; int64_t big; };
    std::vector<GOpt> opts;
    if (Sk <= TN_GATE_MAX_K && Sn <= TN_GATE_MAX_N) opts.push_back({a, b, &st.N, Sa});
    if (Sk <= TN_GATE_MAX_K && Sm <= TN_GATE_MAX_N) opts.push_back({b, a, &st.M, Sb});
    std::sort(opts.begin(), opts.end(), [](const GOpt &x, const GOpt &y) { return x.big > y.big; });
    for (auto &o : opts) {
      std::vector<int> K = k_order(order[o.A], st.K);
      std::vector<int> Nn;
      for (int l : order[o.B]) if (pos_of(*o.N, l) >= 0) Nn.push_back(l);
      GateParams g;
      std::vector<int> ordC;
      if (make_gate(order[o.A], &order[o.B], K, Nn, &g, &ordC)) {
        Loc out = new_tensor(ipow(q, (int)ordC.size()));
        push_gate(g, loc[o.A], &loc[o.B], out, unit[o.B]);
        order[st.c] = ordC;
        loc[st.c] = out;
        return;
      }
    }
    // GEMM path, both role assignments, fewest transposed elements
    GemmChoice c1 = plan_gemm(a, b, st.batch, st.M, st.K, st.N);
    GemmChoice c2 = plan_gemm(b, a, st.batch, st.N, st.K, st.M);
    GemmChoice &ch = (c2.cost < c1.cost || (c2.cost == c1.cost && Sb > Sa)) ? c2 : c1;
    std::vector<int> ordA, ordB;
    Loc LA = loc[ch.A], LB = loc[ch.B];
    if (ch.permA) {
      ordA = ch.bo;
      ordA.insert(ordA.end(), ch.mo.begin(), ch.mo.end());
      ordA.insert(ordA.end(), ch.ko.begin(), ch.ko.end());
      LA = emit_perm(ch.A, ordA);
    } else {
      ordA = order[ch.A];
    }
    if (ch.permB) {
      ordB = ch.bo;
      ordB.insert(ordB.end(), ch.ko.begin(), ch.ko.end());
      ordB.insert(ordB.end(), ch.no.begin(), ch.no.end());
      LB = emit_perm(ch.B, ordB);
    } else {
      ordB = order[ch.B];
    }
    std::vector<int> ordC = ch.bo;
    ordC.insert(ordC.end(), ch.mo.begin(), ch.mo.end());
    ordC.insert(ordC.end(), ch.no.begin(), ch.no.end());
    GemmParams g{};
    g.batch = ipow(q, (int)ch.bo.size());
    g.M = ipow(q, (int)ch.mo.size());
    g.N = ipow(q, (int)ch.no.size());
    g.K = ipow(q, (int)ch.ko.size());
    g.sAb = inner_stride(ordA, ch.bo);
    g.sAm = inner_stride(ordA, ch.mo);
    g.sAk = inner_stride(ordA, ch.ko);
    g.sBb = inner_stride(ordB, ch.bo);
    g.sBk = inner_stride(ordB, ch.ko);
    g.sBn = inner_stride(ordB, ch.no);
    g.sCb = inner_stride(ordC, ch.bo);
    g.sCm = inner_stride(ordC, ch.mo);
    g.sCn = inner_stride(ordC, ch.no);
    Loc out = new_tensor(ipow(q, (int)ordC.size()));
    g.planeA = LA.plane;
    g.planeB = LB.plane;
    g.planeC = out.plane;
    g.P = P;
    pr.gemms.push_back(g);
    Op op;
    op.macs = (double)g.batch * g.M * g.N * g.K;
    op.kind = OP_GEMM;
    op.in0 = LA;
    op.in1 = LB;
    op.out = out;
    op.idx = (int)pr.gemms.size() - 1;
    push(op);
    pr.n_gemm++;
    order[st.c] = ordC;
    loc[st.c] = out;
  }

  bool emit_step(int s) {
    const PStep &st = plan.steps[s];
    if (st.b < 0) return emit_unary(st);
    emit_pair(st);
    return true;
  }

  // ---- fused gate chains
  struct CGate {
    int kind = 0;            // 0 replace, 1 diagonal, 2 contract (ends the chain)
    int pos = -1;            // replaced / contracted position
    int kspin = -1;
    int btensor = -1;
    std::vector<int> bpos;   // positions of B's legs that are legs of the state
    int64_t sBk = 0, sBn = 0, sBb[2] = {0, 0};
  };
  struct Macro {
    bool chain = false;
    int step = -1;
    std::vector<int> steps;
    int in = -1, out = -1;
    std::vector<CGate> gates;
    std::vector<int> touched;   // positions touched by the gates
    std::vector<int> rpos;      // positions replaced by the gates
    // rank-changing ends (folded register chains): the chain starts from the
    // input of a step that adds a leg (the new leg, innermost, is a register
    // leg and gate 0 adds that step's operand) and/or ends with a contraction
    bool grow = false, contract = false;
    std::vector<int> state;     // leg order between the gates
  };
  std::vector<Macro> macros;
  std::vector<int> macro_of;    // tensor -> macro producing it
  bool fuse = true;
  bool regmode = false;         // q == 2 values: register chains (ChainParams mode 1)
  bool fold = true;             // fold diagonal gates into replace tables (values only)
  int kRB = 6;                  // register legs of a register chain (4 to 6; 3 when counting)
  bool grow_inner = false;      // rank-raising chains put the new leg innermost (else slowest)
  int grow_pos(int R) const { return grow_inner ? R - 1 : 0; }
  int tmax = 11, wlow = 5;
  // chains still accepting gates, by the tensor they currently produce; a chain
  // is emitted when a step needs its output as a whole tensor
  std::map<int, Macro> opens;

  int64_t tsize(int t) const { return ipow(q, (int)plan.legset[t].size()); }

  // a rank-preserving step of a big tensor with a small one, as a chain gate
  bool try_gate(const PStep &st, int big, int small, CGate *g) {
    const std::vector<int> &ob = order[big], &os = order[small];
    const int R = (int)ob.size();
    if ((int)os.size() > 3 || R < (regmode ? kRB + 8 : tmax + 3)) return false;
    const std::vector<int> &N = (big == st.a) ? st.N : st.M;
    if (st.K.size() != N.size() || st.K.size() > 1 || st.batch.size() > 2) return false;
    if (regmode && st.K.size() == 1 && st.batch.size() > 1) return false;
    g->btensor = small;
    g->bpos.clear();
    for (int l : st.batch) g->bpos.push_back(pos_of(ob, l));
    for (size_t j = 0; j < st.batch.size(); ++j) g->sBb[j] = stride(os, st.batch[j]);
    if (st.K.size() == 1) {
      g->kind = 0;
      g->pos = pos_of(ob, st.K[0]);
      g->kspin = st.K[0];
      g->sBk = stride(os, st.K[0]);
      g->sBn = stride(os, N[0]);
    } else {
      g->kind = 1;
      g->pos = -1;
      if (g->bpos.empty()) return false;
    }
    return true;
  }

  // Rank-changing steps at the ends of a folded register chain (values, q = 2).
  bool rank_fusion() const { return regmode && fold && P == 0 && kRB >= 5; }

  // a step adding one leg to `big` (no contraction, one batch leg at most): the
  // chain starts from big, the new leg slowest (or innermost with
  // TN_GROW_INNER); gate 0 is the diagonal gate adding the small operand over
  // (new leg, batch leg).  With the new leg slowest the chain, which doubles
  // its tensor, reads and writes each half of the output as one contiguous
  // stream (measured faster than innermost on the square-lattice orders).
  bool try_grow(const PStep &st, int big, int small, CGate *g, std::vector<int> *ord) {
    if (!rank_fusion()) return false;
    const std::vector<int> &ob = order[big], &os = order[small];
    const std::vector<int> &N = (big == st.a) ? st.N : st.M;
    const std::vector<int> &Mb = (big == st.a) ? st.M : st.N;
    (void)Mb;
    if (!st.K.empty() || N.size() != 1 || st.batch.size() > 1) return false;
    if ((int)os.size() != 1 + (int)st.batch.size()) return false;
    const int R = (int)ob.size() + 1;
    if (R < kRB + 8) return false;
    *ord = ob;
    if (grow_inner) ord->push_back(N[0]);
    else ord->insert(ord->begin(), N[0]);
    *g = CGate();
    g->kind = 1;
    g->btensor = small;
    g->bpos.push_back(grow_pos(R));
    g->sBb[0] = stride(os, N[0]);
    if (!st.batch.empty()) {
      g->bpos.push_back(pos_of(*ord, st.batch[0]));
      g->sBb[1] = stride(os, st.batch[0]);
    }
    return true;
  }

  // a step contracting one leg of the open chain's state with a small operand
  // (no new leg, one batch leg at most): the chain's last gate
  // (no new leg, up to two batch legs of which at most one is a register leg of
  // the chain -- the chain ends here, so its register legs are known)
  bool try_contract(const Macro &m, const PStep &st, int big, int small, CGate *g) {
    if (!rank_fusion()) return false;
    const std::vector<int> &ob = order[big], &os = order[small];
    const std::vector<int> &N = (big == st.a) ? st.N : st.M;
    if (st.K.size() != 1 || !N.empty() || st.batch.size() > 2) return false;
    if ((int)os.size() != 1 + (int)st.batch.size()) return false;
    *g = CGate();
    g->kind = 2;
    g->btensor = small;
    g->pos = pos_of(ob, st.K[0]);
    g->kspin = st.K[0];
    g->sBk = stride(os, st.K[0]);
    for (size_t j = 0; j < st.batch.size(); ++j) {
      g->bpos.push_back(pos_of(ob, st.batch[j]));
      g->sBb[j] = stride(os, st.batch[j]);
    }
    if (g->bpos.size() == 2) {
      Macro t = m;
      if (pos_of(t.rpos, g->pos) < 0) t.rpos.push_back(g->pos);
      const std::vector<int> S = reg_legs(t);
      if (pos_of(S, g->bpos[0]) >= 0 && pos_of(S, g->bpos[1]) >= 0) return false;
    }
    return true;
  }

  std::vector<int> local_set(int R, const std::vector<int> &touched) const {
    std::vector<int> T;
    for (int p = std::max(0, R - wlow); p < R; ++p) T.push_back(p);
    for (int p : touched) if (pos_of(T, p) < 0) T.push_back(p);
    std::sort(T.begin(), T.end());
    return T;
  }

  bool fits(const Macro &m, const CGate &g) const {
    if ((int)m.gates.size() >= TN_CHAIN_MAX_G) return false;
    if (regmode) {
      int n = (int)m.rpos.size();
      if ((g.kind == 0 || g.kind == 2) && pos_of(m.rpos, g.pos) < 0) ++n;
      return n <= kRB;
    }
    std::vector<int> t = m.touched;
    if (g.pos >= 0) t.push_back(g.pos);
    for (int p : g.bpos) t.push_back(p);
    const int R = (int)order[m.in].size();
    return (int)local_set(R, t).size() <= tmax;
  }

  void append(Macro &m, int s, const CGate &g, const std::vector<int> *grow_ord = nullptr) {
    const PStep &st = plan.steps[s];
    std::vector<int> ord = grow_ord ? *grow_ord : order[m.out];
    if (g.kind == 0) {
      const std::vector<int> &N = (m.out == st.a) ? st.N : st.M;
      ord[g.pos] = N[0];
      m.touched.push_back(g.pos);
      if (pos_of(m.rpos, g.pos) < 0) m.rpos.push_back(g.pos);
    }
    if (grow_ord) {
      // the new leg is a register leg of the chain
      m.grow = true;
      const int gp = grow_pos((int)ord.size());
      if (pos_of(m.rpos, gp) < 0) m.rpos.push_back(gp);
    }
    m.state = ord;
    if (g.kind == 2) {
      m.contract = true;
      m.touched.push_back(g.pos);
      if (pos_of(m.rpos, g.pos) < 0) m.rpos.push_back(g.pos);
      ord.erase(ord.begin() + g.pos);
    }
    for (int p : g.bpos) m.touched.push_back(p);
    std::sort(m.touched.begin(), m.touched.end());
    m.touched.erase(std::unique(m.touched.begin(), m.touched.end()), m.touched.end());
    m.gates.push_back(g);
    m.steps.push_back(s);
    m.out = st.c;
    order[st.c] = ord;
    const int R = (int)ord.size();
    pr.macs += (double)ipow(q, R) * (g.kind == 0 ? q : 1);
  }

  // register legs of a register chain: the replaced positions (fastest
  // first), padded with the slowest positions to kRB legs
  std::vector<int> reg_legs(const Macro &m) const {
    std::vector<int> S = m.rpos;
    std::sort(S.begin(), S.end(), [](int x, int y) { return x > y; });
    for (int p = 0; (int)S.size() < kRB; ++p)
      if (pos_of(S, p) < 0) S.push_back(p);
    return S;
  }

  ChainParams reg_chain_params(const Macro &m, std::vector<Loc> *blocs) {
    ChainParams cp{};
    // positions are those of the state between the gates; the input lacks the
    // grown leg, the output lacks the contracted one
    const std::vector<int> &ord = m.state.empty() ? order[m.out] : m.state;
    const int R = (int)ord.size();
    std::vector<int> S = reg_legs(m);
    const int kpos = m.contract ? m.gates.back().pos : -1;
    auto s_state = [&](int p) { return int64_t(1) << (R - 1 - p); };
    auto s_in = [&](int p) -> int64_t {
      if (!m.grow) return s_state(p);
      if (p == grow_pos(R)) return 0;
      return grow_inner ? int64_t(1) << (R - 2 - p) : s_state(p);
    };
    auto s_out = [&](int p) -> int64_t {
      if (!m.contract) return s_state(p);
      if (p == kpos) return 0;
      return p < kpos ? int64_t(1) << (R - 2 - p) : s_state(p);
    };
    auto lg = [](int64_t x) { int r = 0; while ((int64_t(1) << r) < x) ++r; return r; };
    cp.mode = 1;
    cp.q = 2;
    cp.t = kRB;          // 6 (values), 3 (values + residue planes)
    cp.tile = 1 << kRB;
    for (int e = 0; e < cp.tile; ++e) {
      int64_t off = 0, oin = 0, oout = 0;
      for (int j = 0; j < kRB; ++j)
        if (e >> j & 1) {
          off += s_state(S[j]);
          oin += s_in(S[j]);
          oout += s_out(S[j]);
        }
      cp.hi_off[e] = off;
      cp.hi_in[e] = oin;
      cp.hi_out[e] = oout;
    }
    std::vector<int64_t> sz, st;
    std::vector<int> sh, inner;   // inner: the segment's fastest position
    for (int p = 0; p < R; ++p) {
      if (pos_of(S, p) >= 0) continue;
      const int64_t sp = s_state(p);
      if (!sz.empty() && p > 0 && pos_of(S, p - 1) < 0) {
        sz.back() *= 2;
        st.back() = sp;
        sh.back()++;
        inner.back() = p;
      } else {
        sz.push_back(2);
        st.push_back(sp);
        sh.push_back(1);
        inner.push_back(p);
      }
    }
    cp.nseg = (int)sz.size();
    cp.outer = int64_t(1) << (R - kRB);
    for (int i = 0; i < cp.nseg; ++i) {
      cp.seg_size[i] = sz[i];
      cp.seg_s[i] = st[i];
      cp.seg_sh[i] = sh[i];
      cp.seg_ssh[i] = lg(st[i]);
      cp.ssh_in[i] = lg(s_in(inner[i]));
      cp.ssh_out[i] = lg(s_out(inner[i]));
    }
    // bit of each outer position in tau: outer positions, fastest first
    std::vector<int> trank(R, -1);
    for (int p = R - 1, r = 0; p >= 0; --p)
      if (pos_of(S, p) < 0) trank[p] = r++;
    cp.ngates = (int)m.gates.size();
    blocs->clear();
    for (int i = 0; i < cp.ngates; ++i) {
      const CGate &g = m.gates[i];
      ChainGate &c = cp.g[i];
      c.kind = g.kind;
      c.ls = (g.kind == 0 || g.kind == 2) ? pos_of(S, g.pos) : 0;
      c.nb = (int)g.bpos.size();
      for (int j = 0; j < c.nb; ++j) {
        c.lsb[j] = pos_of(S, g.bpos[j]);
        c.lsbh[j] = R - 1 - g.bpos[j];
        c.lrank[j] = trank[g.bpos[j]];
        c.sBb[j] = g.sBb[j];
      }
      c.kspin = g.kspin;
      c.sBk = g.sBk;
      c.sBn = g.sBn;
      c.nBel = (int)tsize(g.btensor);
      c.unitB = unit[g.btensor] ? 1 : 0;
      blocs->push_back(loc[g.btensor]);
    }
    cp.P = P;
    if (P == 0 && fold) fold_reg_chain(cp);
    return cp;
  }

  ChainParams chain_params(const Macro &m, std::vector<Loc> *blocs) {
    if (regmode) return reg_chain_params(m, blocs);
    ChainParams cp{};
    const std::vector<int> &ord = order[m.out];
    const int R = (int)ord.size();
    std::vector<int> T = local_set(R, m.touched);
    cp.q = q;
    cp.t = (int)T.size();
    cp.tile = (int)ipow(q, cp.t);
    int w = std::min(R, wlow);
    cp.lo = (int)ipow(q, w);
    cp.nhi = cp.tile / cp.lo;
    cp.loh = 0;
    while ((1 << cp.loh) < cp.lo) ++cp.loh;
    std::vector<int> H(T.begin(), T.end() - w);
    for (int h = 0; h < cp.nhi; ++h) {
      int64_t r = h, off = 0;
      for (int j = (int)H.size() - 1; j >= 0; --j) {
        off += (r % q) * ipow(q, R - 1 - H[j]);
        r /= q;
      }
      cp.hi_off[h] = off;
    }
    // outer positions, merged into runs
    std::vector<int64_t> sz, st;
    for (int p = 0; p < R; ++p) {
      if (pos_of(T, p) >= 0) continue;
      const int64_t sp = ipow(q, R - 1 - p);
      if (!sz.empty() && st.back() == sp * q && p > 0 && pos_of(T, p - 1) < 0) {
        sz.back() *= q;
        st.back() = sp;
      } else {
        sz.push_back(q);
        st.push_back(sp);
      }
    }
    cp.nseg = (int)sz.size();
    cp.outer = 1;
    for (int i = 0; i < cp.nseg; ++i) {
      cp.seg_size[i] = sz[i];
      cp.seg_s[i] = st[i];
      cp.seg_sh[i] = 0;
      while ((int64_t(1) << cp.seg_sh[i]) < sz[i]) cp.seg_sh[i]++;
      cp.outer *= sz[i];
    }
    auto lstride = [&](int p) { return (int)ipow(q, cp.t - 1 - pos_of(T, p)); };
    auto lg = [](int x) { int r = 0; while ((1 << r) < x) ++r; return r; };
    cp.ngates = (int)m.gates.size();
    blocs->clear();
    for (int i = 0; i < cp.ngates; ++i) {
      const CGate &g = m.gates[i];
      ChainGate &c = cp.g[i];
      c.kind = g.kind;
      c.ls = g.kind == 0 ? lstride(g.pos) : 1;
      c.lsh = lg(c.ls);
      c.nb = (int)g.bpos.size();
      for (int j = 0; j < c.nb; ++j) {
        c.lsb[j] = lstride(g.bpos[j]);
        c.lsbh[j] = lg(c.lsb[j]);
        c.sBb[j] = g.sBb[j];
      }
      c.kspin = g.kspin;
      c.sBk = g.sBk;
      c.sBn = g.sBn;
      c.nBel = (int)tsize(g.btensor);
      blocs->push_back(loc[g.btensor]);
    }
    cp.P = P;
    return cp;
  }

  void emit_chain(const Macro &m) {
    std::vector<Loc> bl;
    ChainParams cp = chain_params(m, &bl);
    Loc out = new_tensor(tsize(m.out));
    cp.planeA = loc[m.in].plane;
    cp.planeC = out.plane;
    pr.chains.push_back(cp);
    pr.chain_blocs.push_back(bl);
    Op op;
    op.kind = OP_CHAIN;
    op.in0 = loc[m.in];
    op.out = out;
    op.idx = (int)pr.chains.size() - 1;
    op.macs = 0;
    for (auto &g : m.gates) op.macs += (double)tsize(m.in) * (g.kind == 0 ? q : 1);
    int oi = push(op);
    for (auto &l : bl) use(l, oi);
    pr.n_chain++;
    pr.n_chain_gates += (int)m.gates.size();
    loc[m.out] = out;
  }

  void flush_chain(int out) {
    auto it = opens.find(out);
    if (it == opens.end()) return;
    Macro m = it->second;
    opens.erase(it);
    emit_chain(m);
    macros.push_back(m);
    macro_of[m.out] = (int)macros.size() - 1;
  }

  bool forward() {
    macro_of.assign(plan.legset.size(), -1);
    for (int s = 0; s < (int)plan.steps.size(); ++s) {
      const PStep &st = plan.steps[s];
      if (fuse && st.b >= 0) {
        CGate g;
        const int cur = opens.count(st.a) ? st.a : (opens.count(st.b) ? st.b : -1);
        if (cur >= 0) {
          const int small = st.a == cur ? st.b : st.a;
          flush_chain(small);   // an operand must exist as a whole tensor
          Macro &m = opens[cur];
          if (try_gate(st, cur, small, &g) && fits(m, g)) {
            Macro mm = m;
            opens.erase(cur);
            append(mm, s, g);
            opens[mm.out] = mm;
            continue;
          }
          if (try_contract(m, st, cur, small, &g) && fits(m, g)) {
            Macro mm = m;
            opens.erase(cur);
            append(mm, s, g);   // a contraction ends the chain
            opens[mm.out] = mm;
            flush_chain(mm.out);
            continue;
          }
          flush_chain(cur);
        }
        flush_chain(st.a);
        flush_chain(st.b);
        int big = tsize(st.a) >= tsize(st.b) ? st.a : st.b;
        int small = big == st.a ? st.b : st.a;
        if (try_gate(st, big, small, &g)) {
          Macro m;
          m.chain = true;
          m.in = m.out = big;
          if (fits(m, g)) {
            append(m, s, g);
            opens[m.out] = m;
            continue;
          }
        }
        std::vector<int> gord;
        if (try_grow(st, big, small, &g, &gord)) {
          Macro m;
          m.chain = true;
          m.in = m.out = big;
          append(m, s, g, &gord);
          opens[m.out] = m;
          continue;
        }
      }
      flush_chain(st.a);
      if (st.b >= 0) flush_chain(st.b);
      if (!emit_step(s)) return false;
      Macro m;
      m.step = s;
      m.out = st.c;
      macros.push_back(m);
      macro_of[st.c] = (int)macros.size() - 1;
    }
    while (!opens.empty()) flush_chain(opens.begin()->first);
    return true;
  }

  std::vector<int> macro_inputs(const Macro &m) const {
    std::vector<int> r;
    if (m.chain) {
      r.push_back(m.in);
      for (auto &g : m.gates) r.push_back(g.btensor);
    } else {
      const PStep &st = plan.steps[m.step];
      r.push_back(st.a);
      if (st.b >= 0) r.push_back(st.b);
    }
    return r;
  }

  bool emit_macro(const Macro &m) {
    if (m.chain) {
      emit_chain(m);
      return true;
    }
    return emit_step(m.step);
  }

  // ---- traceback
  std::vector<int> pending;   // macros
  void flush_trace() {
    if (pending.empty()) return;
    Op op;
    op.kind = OP_TRACE;
    op.trace_begin = (int)pr.trace.size();
    op.trace_n = (int)pending.size();
    pr.ops.push_back(op);
    int oi = (int)pr.ops.size() - 1;
    for (int mi : pending) {
      const Macro &m = macros[mi];
      TraceStep t{};
      t.chain = -1;
      if (m.chain) {
        ChainTrace ct{};
        std::vector<Loc> bl;
        ct.p = chain_params(m, &bl);
        // the state between the gates; outer legs are read from the chain's
        // input (without the grown leg, if any)
        const std::vector<int> &ord = m.state.empty() ? order[m.out] : m.state;
        const int R = (int)ord.size();
        std::vector<int> T = regmode ? reg_legs(m) : local_set(R, m.touched);
        for (int p = 0; p < R; ++p) {
          if (pos_of(T, p) >= 0) continue;
          ct.out_spin[ct.nout] = ord[p];
          ct.out_stride[ct.nout] = (m.grow && grow_inner) ? ipow(q, R - 2 - p) : ipow(q, R - 1 - p);
          int rank = 0;   // bit of this outer leg in tau: outer legs faster than it
          for (int p2 = p + 1; p2 < R; ++p2) rank += pos_of(T, p2) < 0;
          ct.out_rank[ct.nout] = rank;
          ct.nout++;
        }
        for (int j = 0; j < (int)T.size(); ++j) ct.local_spin[j] = ord[T[j]];
        t.chain = (int)pr.chain_traces.size();
        pr.chain_traces.push_back(ct);
        pr.ctrace_in.push_back(loc[m.in]);
        pr.ctrace_blocs.push_back(bl);
        pr.trace_smem = std::max(pr.trace_smem, trace_smem_bytes(ct.p, 4));
        use(loc[m.in], oi);
        for (auto &l : bl) use(l, oi);
        pr.trace.push_back(t);
        pr.traceA.push_back(Loc());
        pr.traceB.push_back(Loc());
        continue;
      }
      const PStep &st = plan.steps[m.step];
      const std::vector<int> &oa = order[st.a];
      std::vector<int> K = k_order(oa, st.K);
      t.nk = (int)K.size();
      t.Ks = (int)ipow(q, t.nk);
      for (int j = 0; j < t.nk; ++j) {
        t.k_spin[j] = K[j];
        t.k_sA[j] = stride(oa, K[j]);
        t.k_sB[j] = st.b >= 0 ? stride(order[st.b], K[j]) : 0;
      }
      for (int l : oa)
        if (pos_of(K, l) < 0) {
          t.fa_spin[t.nfa] = l;
          t.fa_stride[t.nfa] = stride(oa, l);
          t.nfa++;
        }
      if (st.b >= 0)
        for (int l : order[st.b])
          if (pos_of(K, l) < 0) {
            t.fb_spin[t.nfb] = l;
            t.fb_stride[t.nfb] = stride(order[st.b], l);
            t.nfb++;
          }
      pr.trace.push_back(t);
      pr.traceA.push_back(loc[st.a]);
      pr.traceB.push_back(st.b >= 0 ? loc[st.b] : Loc());
      use(loc[st.a], oi);
      if (st.b >= 0) use(loc[st.b], oi);
    }
    pending.clear();
  }

  std::vector<char> avail;
  bool recompute(int t) {
    const int mi = macro_of[t];
    if (mi < 0) { err = "recompute: tensor has no producer"; return false; }
    const Macro &m = macros[mi];
    for (int x : macro_inputs(m))
      if (!avail[x] && !recompute(x)) return false;
    if (!emit_macro(m)) return false;
    pr.n_recompute++;
    avail[t] = 1;
    return true;
  }

  bool build(ProgMode mode, int64_t seg_bytes) {
    fuse = std::getenv("TN_NO_FUSION") == nullptr;
    // register chains: q = 2 values, or q = 2 counts with 3 primes + witness
    regmode = q == 2 && (P == 0 || (P == 4 && rb == 8) || (P == 7 && rb == 4)) &&
              std::getenv("TN_TILE_CHAINS") == nullptr;
    fold = std::getenv("TN_NO_FOLD") == nullptr;
    grow_inner = std::getenv("TN_GROW_INNER") != nullptr;
    // values: 6 register legs (2^6 states per thread) with folded tables,
    // 5 for the unfolded gate lists; counts: 3 legs (values + 4 residue planes)
    kRB = fold ? 6 : 5;
    if (const char *rb = std::getenv("TN_REG_BITS")) kRB = std::max(4, std::min(fold ? 6 : 5, std::atoi(rb)));
    if (P > 0) kRB = 3;
    if (q == 3) { tmax = 7; wlow = 4; }
    emit_leaves();
    if (!forward()) return false;
    pr.root = loc[plan.root];
    pr.fwd_end = (int)pr.ops.size();
    if (mode == PM_CONFIG) {
      std::vector<char> stored(plan.legset.size(), 0);
      for (int i = 0; i < plan.n_leaves; ++i) stored[i] = 1;
      std::vector<int64_t> acc(plan.legset.size(), 0);
      for (const Macro &m : macros) {
        int64_t a = tsize(m.out) * 4;
        for (int x : macro_inputs(m))
          if (!stored[x]) a += acc[x];
        acc[m.out] = a;
        if (seg_bytes <= 0 || a > seg_bytes || m.out == plan.root || tsize(m.out) <= 4096)
          stored[m.out] = 1;
      }
      avail = stored;
      for (int mi = (int)macros.size() - 1; mi >= 0; --mi) {
        bool need = false;
        for (int x : macro_inputs(macros[mi])) need = need || !avail[x];
        if (need) {
          flush_trace();
          for (int x : macro_inputs(macros[mi]))
            if (!avail[x] && !recompute(x)) return false;
        }
        pending.push_back(mi);
      }
      flush_trace();
    }
    use(pr.root, (int)pr.ops.size());
    return true;
  }
};

void plan_memory(Program &pr) {
  std::vector<int> idx(pr.bufs.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    return pr.bufs[a].bytes > pr.bufs[b].bytes || (pr.bufs[a].bytes == pr.bufs[b].bytes && a < b);
  });
  std::vector<int> placed;
  int64_t top = 0;
  for (int i : idx) {
    BufInfo &b = pr.bufs[i];
    if (b.last < 0) { b.first = b.last = 0; }
    std::vector<std::pair<int64_t, int64_t>> busy;
    for (int j : placed) {
      const BufInfo &o = pr.bufs[j];
      if (o.first <= b.last && b.first <= o.last) busy.push_back({o.off, o.off + o.bytes});
    }
    std::sort(busy.begin(), busy.end());
    int64_t off = 0;
    for (auto &r : busy) {
      if (r.first >= off + b.bytes) break;
      off = std::max(off, r.second);
    }
    b.off = off;
    top = std::max(top, off + b.bytes);
    placed.push_back(i);
  }
  pr.arena_bytes = std::max<int64_t>(top, kAlign);
}

}  // namespace

int64_t abs_off(const Program &pr, const Loc &l) { return pr.bufs[l.buf].off + l.xoff; }

bool build_program(const Net &net, const Plan &plan, ProgMode mode, Dtype dt, int P,
                   int64_t seg_bytes, Program *pr, std::string *err, int rbytes) {
  *pr = Program();
  pr->mode = mode;
  pr->dt = dt;
  pr->q = net.q;
  pr->P = P;
  if (rbytes != 4 && rbytes != 8) {
    *err = "residue width must be 4 or 8 bytes";
    return false;
  }
  pr->rbytes = rbytes;
  Builder bd(net, plan, *pr);
  if (!bd.build(mode, seg_bytes)) {
    *err = bd.err.empty() ? "program: lowering failed" : bd.err;
    return false;
  }
  plan_memory(*pr);
  if (const char *dump = std::getenv("TN_DUMP_PROGRAM")) {
    // "1": every program built; "c": only traceback / counting programs
    if (*dump == '1' || (*dump == 'c' && mode != PM_ENERGY)) {
      std::fprintf(stderr, "program mode %d ops %zu\n", (int)mode, pr->ops.size());
      for (size_t i = 0; i < pr->ops.size(); ++i) {
        const Op &o = pr->ops[i];
        std::fprintf(stderr, "op %zu kind %d bytes %.0f in0 %lld in1 %lld out %lld", i, (int)o.kind,
                     o.bytes,
                     (long long)(o.in0.buf >= 0 ? o.in0.plane : -1),
                     (long long)(o.in1.buf >= 0 ? o.in1.plane : -1),
                     (long long)(o.out.buf >= 0 ? o.out.plane : -1));
        if (o.kind == OP_GATE) {
          const GateParams &g = pr->gates[o.idx];
          std::fprintf(stderr, " outer %lld Ks %d Ns %d nseg %d inA %d outA %d", (long long)g.outer,
                       g.Ks, g.Ns, g.nseg, o.in0.buf, o.out.buf);
          for (int s2 = 0; s2 < g.nseg; ++s2)
            std::fprintf(stderr, " [%lld:%lld,%lld,%lld]", (long long)g.seg_size[s2],
                         (long long)g.seg_sA[s2], (long long)g.seg_sB[s2], (long long)g.seg_sC[s2]);
          std::fprintf(stderr, " kA");
          for (int k = 0; k < g.Ks; ++k) std::fprintf(stderr, " %lld", (long long)g.kA[k]);
          std::fprintf(stderr, " nC");
          for (int k = 0; k < g.Ns; ++k) std::fprintf(stderr, " %lld", (long long)g.nC[k]);
        }
        if (o.kind == OP_CHAIN) {
          const ChainParams &c = pr->chains[o.idx];
          std::fprintf(stderr, " chain mode %d outer %lld t %d", c.mode, (long long)c.outer, c.t);
          if (c.mode == 1) {
            // memory position (log2 of the element offset) of each register leg
            // in the input and the output layout (-1: not a leg there)
            for (int side = 0; side < 2; ++side) {
              std::fprintf(stderr, side ? " rout" : " rin");
              for (int b = 0; b < c.t; ++b) {
                const int64_t o = side ? c.hi_out[1 << b] : c.hi_in[1 << b];
                int q = -1;
                if (o > 0) for (q = 0; (int64_t(1) << q) < o; ++q) {}
                std::fprintf(stderr, " %d", q);
              }
            }
          }
          std::fprintf(stderr, " gates");
          for (int g = 0; g < c.ngates; ++g)
            std::fprintf(stderr, " (%d,%d,%d,%d,%d)", c.g[g].kind, c.g[g].ls, c.g[g].nb, c.g[g].lsb[0],
                         c.g[g].nb > 1 ? c.g[g].lsb[1] : 9);
        }
        if (o.kind == OP_GEMM) {
          const GemmParams &g = pr->gemms[o.idx];
          std::fprintf(stderr, " b %lld M %lld N %lld K %lld", (long long)g.batch, (long long)g.M,
                       (long long)g.N, (long long)g.K);
        }
        std::fprintf(stderr, "\n");
      }
    }
  }
  // absolute offsets of leaves and traceback operands
  const int64_t lbase = pr->bufs[pr->leaves_loc.buf].off;
  for (int i = 0; i < plan.n_leaves; ++i) {
    const Net::Leaf &L = net.leaves[i];
    LeafDesc d{};
    d.off_x = lbase + pr->leaves_loc.xoff + pr->leaf_elem[i] * 4;
    d.off_n = lbase + pr->leaves_loc.noff + pr->leaf_elem[i] * pr->rbytes;
    d.plane = pr->leaves_loc.plane;
    d.kind = L.kind;
    d.edge = L.edge;
    if (L.kind == 0) {
      // memory legs are (min, max); map the absorbed fields accordingly
      bool sw = L.u > L.v;
      d.u = sw ? L.v : L.u;
      d.v = sw ? L.u : L.v;
      d.fu = sw ? L.fv : L.fu;
      d.fv = sw ? L.fu : L.fv;
    } else {
      d.u = L.u;
      d.v = -1;
      d.fu = L.fu;
      d.fv = 0;
    }
    pr->leaves.push_back(d);
  }
  for (size_t i = 0; i < pr->trace.size(); ++i) {
    if (pr->trace[i].chain >= 0) continue;
    pr->trace[i].offA = abs_off(*pr, pr->traceA[i]) / 4;
    pr->trace[i].offB = pr->traceB[i].buf >= 0 ? abs_off(*pr, pr->traceB[i]) / 4 : -1;
  }
  auto patch = [&](ChainParams &cp, const std::vector<Loc> &bl) {
    for (int g = 0; g < cp.ngates; ++g) {
      cp.g[g].offB = abs_off(*pr, bl[g]) / 4;
      cp.g[g].offBn = (pr->bufs[bl[g].buf].off + bl[g].noff) / pr->rbytes;
      cp.g[g].planeB = bl[g].plane;
    }
  };
  for (size_t i = 0; i < pr->chains.size(); ++i) patch(pr->chains[i], pr->chain_blocs[i]);
  for (size_t i = 0; i < pr->chain_traces.size(); ++i) {
    patch(pr->chain_traces[i].p, pr->ctrace_blocs[i]);
    pr->chain_traces[i].offIn = abs_off(*pr, pr->ctrace_in[i]) / 4;
  }
  return true;
}

}  // namespace tn
