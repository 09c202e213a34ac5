// planner.cpp -- network leaves, contraction orders and step classification.
//
// The network (Sec. II): one bond tensor per edge holding the negative bond
// energy; each spin is a shared index (hyperedge) of every tensor touching it,
// which is the tropical copy tensor of Sec. II without materialising it; the
// field of a spin (the vertex tensor diag(h, -h)) is folded into the first
// bond that touches the spin, or into a one-leg leaf for an isolated spin.
//
// Orders (Sec. III): a spin-elimination sweep (the row-by-row circuit sweep of
// Fig. 1b for lattices) or a randomized greedy pair selection.
#include "planner.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <queue>
#include <random>
#include <set>
#include <thread>

namespace tn {

void Net::build_leaves() {
  leaves.clear();
  std::vector<int> deg(n, 0);
  for (int e = 0; e < m; ++e) { deg[eu[e]]++; deg[ev[e]]++; }
  std::vector<char> field_done(n, 0);
  const bool hasf = !h.empty();
  for (int e = 0; e < m; ++e) {
    Leaf L{0, e, eu[e], ev[e], 0, 0};
    if (hasf) {
      if (!field_done[eu[e]]) { L.fu = 1; field_done[eu[e]] = 1; }
      if (!field_done[ev[e]]) { L.fv = 1; field_done[ev[e]] = 1; }
    }
    leaves.push_back(L);
  }
  for (int i = 0; i < n; ++i)
    if (deg[i] == 0) leaves.push_back(Leaf{1, -1, i, -1, hasf ? 1 : 0, 0});
}

double CostModel::step_time(double in_bytes, double out_bytes, double macs) const {
  return std::max((in_bytes + out_bytes) / bytes_per_s, macs / macs_per_s) + launch_s;
}

namespace {

// Live-tensor bookkeeping shared by the order finders.
struct Sim {
  int q;
  std::vector<std::vector<int>> legs;
  std::vector<char> alive;
  std::vector<int> count;  // live tensors holding each spin
  Tree *tree;

  Sim(const Net &net, Tree *t) : q(net.q), count(net.n, 0), tree(t) {
    for (auto &L : net.leaves) {
      std::vector<int> l;
      if (L.kind == 0) l = {std::min(L.u, L.v), std::max(L.u, L.v)};
      else l = {L.u};
      for (int s : l) count[s]++;
      legs.push_back(l);
      alive.push_back(1);
    }
  }
  // legs of the merge of a and b (contracted and reduced legs dropped)
  std::vector<int> out_legs(int a, int b) const {
    const auto &A = legs[a], &B = legs[b];
    std::vector<int> o;
    size_t i = 0, j = 0;
    while (i < A.size() || j < B.size()) {
      if (j == B.size() || (i < A.size() && A[i] < B[j])) {
        if (count[A[i]] > 1) o.push_back(A[i]);
        ++i;
      } else if (i == A.size() || B[j] < A[i]) {
        if (count[B[j]] > 1) o.push_back(B[j]);
        ++j;
      } else {
        if (count[A[i]] > 2) o.push_back(A[i]);
        ++i; ++j;
      }
    }
    return o;
  }
  int merge(int a, int b) {
    std::vector<int> o = out_legs(a, b);
    for (int s : legs[a]) count[s]--;
    for (int s : legs[b]) count[s]--;
    for (int s : o) count[s]++;
    alive[a] = alive[b] = 0;
    legs.push_back(o);
    alive.push_back(1);
    tree->steps.push_back({a, b});
    return (int)legs.size() - 1;
  }
  int reduce(int a) {
    std::vector<int> o;
    for (int s : legs[a]) if (count[s] > 1) o.push_back(s);
    for (int s : legs[a]) count[s]--;
    for (int s : o) count[s]++;
    alive[a] = 0;
    legs.push_back(o);
    alive.push_back(1);
    tree->steps.push_back({a, -1});
    return (int)legs.size() - 1;
  }
  // merge every remaining live tensor, smallest first
  void finish() {
    for (;;) {
      std::vector<int> live;
      for (int i = 0; i < (int)legs.size(); ++i) if (alive[i]) live.push_back(i);
      if (live.size() <= 1) return;
      std::sort(live.begin(), live.end(), [&](int x, int y) {
        return legs[x].size() < legs[y].size() || (legs[x].size() == legs[y].size() && x < y);
      });
      merge(live[0], live[1]);
    }
  }
};

}  // namespace

bool tree_from_sweep(const Net &net, const std::vector<int> &seq, Tree *t, std::string *err) {
  t->steps.clear();
  std::vector<char> seen(net.n, 0);
  std::vector<int> order;
  for (int v : seq) {
    if (v < 0 || v >= net.n) { *err = "sweep: spin id out of range"; return false; }
    if (seen[v]) { *err = "sweep: spin repeated"; return false; }
    seen[v] = 1;
    order.push_back(v);
  }
  for (int v = 0; v < net.n; ++v) if (!seen[v]) order.push_back(v);
  Sim sim(net, t);
  // holders of each spin, maintained lazily
  for (int v : order) {
    for (;;) {
      std::vector<int> hold;
      for (int i = 0; i < (int)sim.legs.size(); ++i)
        if (sim.alive[i] && std::binary_search(sim.legs[i].begin(), sim.legs[i].end(), v))
          hold.push_back(i);
      if (hold.empty()) break;
      if (hold.size() == 1) {
        if (sim.count[v] == 1) sim.reduce(hold[0]);
        break;
      }
      std::sort(hold.begin(), hold.end(), [&](int x, int y) {
        return sim.legs[x].size() < sim.legs[y].size() ||
               (sim.legs[x].size() == sim.legs[y].size() && x < y);
      });
      sim.merge(hold[0], hold[1]);
    }
  }
  sim.finish();
  return true;
}

namespace {

double signlog(double c) { return c >= 0 ? std::log2(c + 1.0) : -std::log2(-c + 1.0); }

bool greedy_once(const Net &net, std::mt19937_64 &rng, double temp, double alpha, Tree *t) {
  t->steps.clear();
  Sim sim(net, t);
  const double q = net.q;
  std::vector<std::vector<int>> where(net.n);
  for (int i = 0; i < (int)sim.legs.size(); ++i)
    for (int s : sim.legs[i]) where[s].push_back(i);
  std::uniform_real_distribution<double> U(1e-12, 1.0);
  auto score = [&](int a, int b) {
    double so = std::pow(q, (double)sim.out_legs(a, b).size());
    double sa = std::pow(q, (double)sim.legs[a].size());
    double sb = std::pow(q, (double)sim.legs[b].size());
    double s = signlog(so - alpha * (sa + sb));
    if (temp > 0) s -= temp * (-std::log(-std::log(U(rng))));
    return s;
  };
  typedef std::tuple<double, int, int> Cand;
  std::priority_queue<Cand, std::vector<Cand>, std::greater<Cand>> heap;
  std::set<std::pair<int, int>> pushed;
  auto push_pairs_of = [&](int a) {
    for (int s : sim.legs[a])
      for (int b : where[s]) {
        if (b == a || !sim.alive[b]) continue;
        auto key = std::make_pair(std::min(a, b), std::max(a, b));
        if (pushed.insert(key).second) heap.push(Cand(score(key.first, key.second), key.first, key.second));
      }
  };
  for (int i = 0; i < (int)sim.legs.size(); ++i) push_pairs_of(i);
  while (!heap.empty()) {
    Cand c = heap.top();
    heap.pop();
    int a = std::get<1>(c), b = std::get<2>(c);
    if (!sim.alive[a] || !sim.alive[b]) continue;
    int id = sim.merge(a, b);
    for (int s : sim.legs[id]) where[s].push_back(id);
    push_pairs_of(id);
  }
  sim.finish();
  return true;
}

}  // namespace

double plan_cost(const Plan &p, int q, const CostModel &cm) {
  double tot = 0;
  for (auto &s : p.steps) {
    double sa = std::pow((double)q, (double)p.legset[s.a].size());
    double sb = s.b >= 0 ? std::pow((double)q, (double)p.legset[s.b].size()) : 0;
    double sc = std::pow((double)q, (double)p.legset[s.c].size());
    double macs = sc * std::pow((double)q, (double)s.K.size());
    tot += cm.step_time(4 * (sa + sb), 4 * sc, macs);
  }
  return tot;
}

bool tree_greedy(const Net &net, uint64_t seed, int restarts, const CostModel &cm, Tree *t,
                 std::string *err, const std::function<double(const Plan &)> &score) {
  if (restarts < 1) restarts = 1;
  // restart r draws (temperature, cost weight) and its own generator from the
  // seed alone, so the result does not depend on how restarts are spread over
  // host threads
  std::vector<double> temp(restarts, 0.0), alpha(restarts, 1.0);
  {
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    for (int r = 1; r < restarts; ++r) {
      temp[r] = std::exp(std::log(1e-3) + U(rng) * (std::log(1.0) - std::log(1e-3)));
      alpha[r] = std::exp(std::log(0.1) + U(rng) * (std::log(4.0) - std::log(0.1)));
    }
  }
  std::vector<double> cost(restarts, INFINITY);
  std::vector<Tree> trees(restarts);
  std::vector<std::string> errs(restarts);
  std::atomic<int> next(0);
  auto worker = [&]() {
    for (;;) {
      const int r = next.fetch_add(1);
      if (r >= restarts) return;
      std::mt19937_64 rng(seed * 0x9E3779B97F4A7C15ull + (uint64_t)r * 0xBF58476D1CE4E5B9ull + 1);
      greedy_once(net, rng, temp[r], alpha[r], &trees[r]);
      Plan p;
      if (!classify(net, trees[r], &p, &errs[r])) continue;
      if (p.log2_peak > 34.0) continue;
      cost[r] = score ? score(p) : plan_cost(p, net.q, cm);
    }
  };
  unsigned nth = std::thread::hardware_concurrency();
  if (nth == 0) nth = 1;
  nth = std::min<unsigned>(nth, 32);
  nth = std::min<unsigned>(nth, (unsigned)restarts);
  std::vector<std::thread> pool;
  for (unsigned i = 1; i < nth; ++i) pool.emplace_back(worker);
  worker();
  for (auto &th : pool) th.join();
  int best = -1;
  for (int r = 0; r < restarts; ++r) {
    if (!errs[r].empty()) { *err = errs[r]; return false; }
    if (std::isfinite(cost[r]) && (best < 0 || cost[r] < cost[best])) best = r;
  }
  if (best < 0) { *err = "greedy: every tree exceeds 2^34 elements"; return false; }
  *t = trees[best];
  return true;
}

bool classify(const Net &net, const Tree &t, Plan *plan, std::string *err) {
  Plan &P = *plan;
  P = Plan();
  const int L = (int)net.leaves.size();
  P.n_leaves = L;
  std::vector<int> count(net.n, 0);
  std::vector<char> alive;
  for (auto &lf : net.leaves) {
    std::vector<int> l;
    if (lf.kind == 0) l = {std::min(lf.u, lf.v), std::max(lf.u, lf.v)};
    else l = {lf.u};
    for (int s : l) count[s]++;
    P.legset.push_back(l);
    P.producer.push_back(-1);
    alive.push_back(1);
  }
  std::vector<int> ext2int(L);
  for (int i = 0; i < L; ++i) ext2int[i] = i;
  double ops = 0;

  auto newt = [&](const std::vector<int> &legs, int step) {
    P.legset.push_back(legs);
    P.producer.push_back(step);
    alive.push_back(1);
    return (int)P.legset.size() - 1;
  };
  auto do_reduce = [&](int a) {
    PStep s;
    s.a = a; s.b = -1;
    for (int l : P.legset[a]) (count[l] == 1 ? s.K : s.M).push_back(l);
    for (int l : s.K) count[l] = 0;
    alive[a] = 0;
    s.c = newt(s.M, (int)P.steps.size());
    ops += std::pow((double)net.q, (double)(s.M.size() + s.K.size()));
    P.steps.push_back(s);
    return s.c;
  };
  auto has_single = [&](int a) {
    for (int l : P.legset[a]) if (count[l] == 1) return true;
    return false;
  };

  for (auto &st : t.steps) {
    int ea = st.first, eb = st.second;
    int next_ext = (int)ext2int.size();
    if (ea < 0 || ea >= next_ext || eb >= next_ext || eb < -1 || ea == eb) {
      *err = "tree: step refers to an unknown tensor";
      return false;
    }
    int a = ext2int[ea];
    if (!alive[a]) { *err = "tree: tensor used twice"; return false; }
    if (eb == -1) {
      ext2int.push_back(do_reduce(a));
      continue;
    }
    int b = ext2int[eb];
    if (!alive[b]) { *err = "tree: tensor used twice"; return false; }
    if (has_single(a)) a = do_reduce(a);
    if (has_single(b)) b = do_reduce(b);
    PStep s;
    s.a = a; s.b = b;
    const auto &A = P.legset[a], &B = P.legset[b];
    for (int l : A) {
      if (std::binary_search(B.begin(), B.end(), l)) (count[l] > 2 ? s.batch : s.K).push_back(l);
      else s.M.push_back(l);
    }
    for (int l : B) if (!std::binary_search(A.begin(), A.end(), l)) s.N.push_back(l);
    for (int l : s.K) count[l] = 0;
    for (int l : s.batch) count[l]--;
    std::vector<int> out = s.batch;
    out.insert(out.end(), s.M.begin(), s.M.end());
    out.insert(out.end(), s.N.begin(), s.N.end());
    std::sort(out.begin(), out.end());
    alive[a] = alive[b] = 0;
    s.c = newt(out, (int)P.steps.size());
    ops += std::pow((double)net.q, (double)(s.batch.size() + s.M.size() + s.N.size() + s.K.size()));
    P.steps.push_back(s);
    ext2int.push_back(s.c);
  }
  int root = -1, nalive = 0;
  for (int i = 0; i < (int)alive.size(); ++i) if (alive[i]) { root = i; nalive++; }
  if (nalive != 1) { *err = "tree: does not merge every tensor into one root"; return false; }
  if (!P.legset[root].empty()) root = do_reduce(root);
  if (!P.legset[root].empty()) { *err = "tree: root keeps open legs"; return false; }
  P.root = root;
  P.consumer.assign(P.legset.size(), -1);
  for (int i = 0; i < (int)P.steps.size(); ++i) {
    P.consumer[P.steps[i].a] = i;
    if (P.steps[i].b >= 0) P.consumer[P.steps[i].b] = i;
  }
  size_t peak = 0;
  for (auto &l : P.legset) peak = std::max(peak, l.size());
  P.log2_peak = peak * std::log2((double)net.q);
  P.log2_ops = ops > 0 ? std::log2(ops) : 0;
  return true;
}

}  // namespace tn
