// sampler.h -- uniform sampling of ground states by conditional counts.
//
// Sec. III: besides backtracking, ground states can be drawn by fixing the
// spins one at a time in an arbitrary order, each with its conditional
// probability of being in a ground state given the spins fixed before it.
// With exact degeneracy counts this gives every ground state the same
// probability 1/count.
//
// Conditioning uses fields.  Add a field p_j in {+1, -1} to every fixed spin
// j (k of them).  A state agreeing with all k pins has E' = E - k; one that
// disagrees on at least one has E' >= E - (k - 2).  So the pinned instance
// has minimum E_min - k exactly when some ground state agrees with the pins,
// and then its minimisers are exactly those ground states: its count is the
// number of ground states with that prefix.  (Any positive pin strength
// works; 1 keeps integral instances integral and exact.)
//
// This file is host logic only: the counts come from a callback (the library
// passes batched GPU contractions, the host tests pass brute force).
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace tn {

// Unsigned big integer, little-endian 64-bit limbs (no leading-zero limbs
// required).
typedef std::vector<uint64_t> Big;

// Counts K pinned instances.  h holds K field vectors of n floats each; on
// success E[k] is the minimum energy and cnt[k] the number of minimisers of
// instance k.  Returns 0, or a nonzero status that the sampler passes on.
typedef std::function<int(const std::vector<float> &h, int K, std::vector<double> *E,
                          std::vector<Big> *cnt)>
    CountFn;

// Draw S ground states of an Ising instance with n spins and fields h0
// (zeros when it has none), fixing spins in `order` (a permutation of
// 0..n-1).  At most `chunk` samples share one batch of 2 * chunk counts.
// sigma: S * n values +-1, sample-major.  Sample s draws its random numbers
// from a counter-based generator keyed by (seed, s, step), so a sample does
// not depend on S or chunk.  Returns 0 or the callback's status; *err says
// why (a status of -1 means the counts were inconsistent).
int sample_ground_states(int n, int S, const std::vector<int> &order, const std::vector<float> &h0,
                         uint64_t seed, int chunk, const CountFn &count,
                         std::vector<int8_t> *sigma, std::string *err);

// Helpers (exposed for tests).
uint64_t mix64(uint64_t x);                         // SplitMix64 finaliser
bool big_less(const Big &a, const Big &b);
Big big_add(const Big &a, const Big &b);
Big uniform_below(const Big &bound, uint64_t seed, uint64_t s, uint64_t step);

}  // namespace tn
