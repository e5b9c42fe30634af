// Tensor networks of circuits (step (a) of Sec. 3.2), contraction paths and
// slicing (steps (c) and (d)).  Host-side data structures.
#pragma once

#include <cstdint>
#include <functional>
#include <memory>
#include <vector>

#include "tdq_internal.h"

namespace tdq {

enum LeafKind : int {
  LEAF_KET0 = 0,  // |0>: one index
  LEAF_GATE = 1,  // gate tensor (conj for the bra network): indices (outs..., ins...)
  LEAF_OBS_Z = 2, // Z between ket and bra legs: indices (bra, ket)
  LEAF_BIT = 3,   // <b| (amplitude read-out) or <0|^* closing the bra: one index
  LEAF_HALF0 = 4, // first-qubit half of a split block-diagonal gate: (bond, out, in) = [out == in == bond]
  LEAF_HALF1 = 5, // second-qubit half: (bond, out, in) = V_bond[out][in]
  LEAF_DIAG = 6,  // diagonal reduction (hyper networks): a diagonal gate (Z, RZ on one
                  // index; CZ, RZZ on two) or the Z observable as its diagonal, the
                  // qubit wires passing through as hyperedges; anti-diagonal
                  // reduction: the phases M[1-i][i] of a Y gate on its input index
  LEAF_CTRL = 7,  // CNOT with its control wire as a hyperedge: (c, out, in) = [out == in xor c]
};

struct Leaf {
  int kind = 0;
  int gate = -1;  // circuit gate index for LEAF_GATE
  int conj = 0;   // bra-side copy: entries conjugated
  int bit = 0;    // LEAF_BIT value
  int flip = 0;   // bit a set: index a is read complemented (the entry at index
                  // value v is the plain tensor's entry at v ^ 1) -- the wire
                  // passed an odd number of anti-diagonal gates (X, Y) that the
                  // hyper network reduced away
  std::vector<int> idx;
};

struct Network {
  tdq_circuit circ;        // copy of the circuit (angles are read from it)
  std::vector<Leaf> leaves;
  int n_indices = 0;
  int output = 0;          // TDQ_OUT_EXPVAL (one term) or TDQ_OUT_AMPLITUDE
  int which = 0;           // term or amplitude index
  int split = 0;           // block-diagonal two-qubit gates split into two halves
  int hyper = 0;           // diagonal reduction: indices may be shared by more than two tensors
  double coeff = 1.0;      // term coefficient (expectation networks)
  int qubits_kept = 0, gates_kept = 0;
};

// One pairwise contraction of the SSA path: tensors a and b (ids < n_leaves
// are leaves, id n_leaves + s is the result of step s).
struct Step {
  int a, b;
};

struct Plan {
  std::shared_ptr<Network> net;
  std::vector<Step> steps;
  std::vector<int> sliced;  // sliced index ids
  double log2_flops = 0;    // per slice, whole path (complex MACs counted as p(2q-1))
  double flops = 0;         // all slices
  int max_log2_width = 0;   // per slice
  double log2_bytes = 0;
};

// xoshiro256** (Blackman and Vigna), seeded by splitmix64
struct Rng {
  uint64_t s[4];
  explicit Rng(uint64_t seed) {
    for (int i = 0; i < 4; i++) {
      seed += 0x9e3779b97f4a7c15ull;
      uint64_t z = seed;
      z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
      z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
      s[i] = z ^ (z >> 31);
    }
  }
  static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
  uint64_t next() {
    const uint64_t r = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return r;
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Live holder counts of every index at the start of a path: the tensors that
// hold it, plus one for an index held by a single tensor (an open index,
// which no contraction may sum).
std::vector<int> live_counts(const Network& net);
// Indices of the tensor that contracting a and b gives when live[i] tensors
// (a and b among them) hold index i: an index stays while a tensor other than
// a and b holds it -- a hyperedge continuing elsewhere -- and is summed
// otherwise (then it is on both a and b).  Order: a's kept indices, then b's
// not on a.  With every index on exactly two tensors this is the symmetric
// difference.  *n_summed (if given) = indices summed.
std::vector<int> merge_live(const std::vector<int>& a, const std::vector<int>& b, const std::vector<int>& live,
                            int* n_summed);
// greedy / random-greedy path over the tensors T0 (Sec. 3.2.2); live[i] counts
// every holder of index i, those outside T0 included (live_counts order)
std::vector<Step> greedy_path_sets(const std::vector<std::vector<int>>& T0, const std::vector<int>& live,
                                   double temperature, uint64_t seed);

// index sets of every SSA tensor after removing `sliced`; with `summed`, also
// the number of indices each step sums
std::vector<std::vector<int>> ssa_indices(const Network& net, const std::vector<Step>& steps,
                                          const std::vector<int>& sliced, std::vector<int>* summed = nullptr);
void plan_measure(Plan& p);

// Contraction tree by recursive bipartition of the network's hypergraph
// (Sec. 3.2.2), read bottom-up into a pairwise path; the trial's
// hyper-parameters (imbalance, outer-index weight, greedy cutoff) are drawn
// from `seed`.
std::vector<Step> partition_tree(const Network& net, uint64_t seed);
// The sliced index set with the fewest FLOPs over all slices among `trials`
// randomised greedy slicings (Sec. 3.2.3) of the path to 2^target entries per
// tensor; trial 0 is the plain greedy rule, and `incumbent` (if given) competes.
std::vector<int> best_slices(const Network& net, const std::vector<Step>& steps, int target, int trials,
                             uint64_t seed, const std::vector<int>* incumbent, bool threads);
// Rank simplification (Sec. 3.2.1): the contractions that do not widen the
// network, as the first steps of a path; `rest` gets the SSA ids left.
std::vector<Step> rank_simplify(const Network& net, std::vector<int>& rest);
// fn(k) for k in [0, n) on the host's cores
void parallel_trials(int n, const std::function<void(int)>& fn);

}  // namespace tdq

struct tdq_network {
  std::shared_ptr<tdq::Network> net;
};

struct tdq_plan {
  tdq::Plan plan;
};
