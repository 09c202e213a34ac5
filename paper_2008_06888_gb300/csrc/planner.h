// planner.h -- host-side network construction, contraction orders and step
// classification (the pairwise contraction tree of Sec. III).
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace tn {

// The spin glass of Eq. 1 (q = 2) or the Potts glass of App. C (q = 3).
struct Net {
  int n = 0, q = 2, m = 0;
  std::vector<int> eu, ev;        // edges
  std::vector<float> J, h;        // h empty: no fields
  // leaves: one per edge (legs u, v) then one per isolated spin (leg u)
  struct Leaf { int kind, edge, u, v, fu, fv; };
  std::vector<Leaf> leaves;
  void build_leaves();
};

// A contraction tree over tensor ids: leaves are 0..L-1, step s creates
// tensor L + s.  b == -1 marks a unary reduction of every leg of a that no
// other live tensor holds.
struct Tree {
  std::vector<std::pair<int, int>> steps;
};

// One classified step.  Pairwise: C = A (.) B with
//   batch: legs in A and B still held by a third tensor,
//   K:     legs in A and B held by no other tensor (contracted, Sec. III),
//   M / N: legs only in A / only in B that other tensors still hold.
// Unary (b == -1): K = legs of A held by nothing else, M = the rest.
struct PStep {
  int a, b, c;
  std::vector<int> batch, M, K, N;
};

struct Plan {
  int n_leaves = 0;
  std::vector<std::vector<int>> legset;   // per tensor, sorted spin ids
  std::vector<int> producer;              // step creating the tensor, -1 leaf
  std::vector<int> consumer;              // step consuming the tensor, -1 root
  std::vector<PStep> steps;
  int root = -1;
  double log2_peak = 0, log2_ops = 0;
};

// Cost model of one GB300 (used to rank candidate trees).
struct CostModel {
  double bytes_per_s = 6.0e12;     // HBM copy bandwidth
  double macs_per_s = 1.5e13;      // tropical multiply-adds on the CUDA cores
  double launch_s = 3.0e-6;
  double step_time(double in_bytes, double out_bytes, double macs) const;
};

// Spin-elimination order -> tree (every tensor holding the spin is merged,
// smallest first, which contracts the spin).
bool tree_from_sweep(const Net &net, const std::vector<int> &seq, Tree *t, std::string *err);
// Randomized greedy (log-size score with Gumbel noise), best of `restarts`.
// `score` (optional) ranks a classified candidate (lower is better); without it
// the per-step cost model is used.
bool tree_greedy(const Net &net, uint64_t seed, int restarts, const CostModel &cm, Tree *t,
                 std::string *err, const std::function<double(const Plan &)> &score = nullptr);
// Validate a user tree and classify every step (inserts unary reductions).
bool classify(const Net &net, const Tree &t, Plan *plan, std::string *err);
double plan_cost(const Plan &p, int q, const CostModel &cm);

}  // namespace tn
