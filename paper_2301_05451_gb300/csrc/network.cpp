// Step (a) of Sec. 3.2: the tensor network of a circuit's output, with the
// light-cone reduction of expectation networks; steps (c)-(d): greedy and
// random-greedy pairwise paths ranked by the FLOP count p(2q-1) of Sec.
// 3.2.2, greedy index slicing (Sec. 3.2.3), and the trial loop that picks the
// path (greedy, random-greedy or hypergraph partition) and slicing with the
// fewest FLOPs over all slices.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <queue>
#include <set>
#include <string>

#include "network.h"

namespace tdq {

// ------------------------------------------------------------------ builder

static int build_network(const tdq_circuit* c, int output, int which, int lightcone, int split, int hyper,
                         Network& N) {
  N.circ = *c;
  N.split = split;
  N.hyper = hyper;
  N.output = output;
  N.which = which;
  const int n = c->n;
  std::vector<int> kept;
  std::vector<char> inq(n, 0);
  if (output == TDQ_OUT_EXPVAL) {
    const Term& t = c->terms[which];
    N.coeff = t.coeff;
    for (int q : t.zq) inq[q] = 1;
    if (lightcone) {
      // backward causal cone: keep a gate iff it touches the cone, then its
      // qubits join the cone; the others cancel against their conjugates
      for (int g = (int)c->gates.size() - 1; g >= 0; g--) {
        const GateRec& G = c->gates[g];
        const int ar = gate_arity(G.kind);
        bool touch = inq[G.q[0]] || (ar == 2 && inq[G.q[1]]);
        if (!touch) continue;
        kept.push_back(g);
        inq[G.q[0]] = 1;
        if (ar == 2) inq[G.q[1]] = 1;
      }
      std::reverse(kept.begin(), kept.end());
    } else {
      for (int g = 0; g < (int)c->gates.size(); g++) kept.push_back(g);
      std::fill(inq.begin(), inq.end(), 1);
    }
  } else {
    for (int g = 0; g < (int)c->gates.size(); g++) kept.push_back(g);
    std::fill(inq.begin(), inq.end(), 1);
  }
  int next = 0;
  std::vector<int> w(n, -1);
  // anti-diagonal reduction (hyper networks): X and Y gates keep the wire's
  // index and mark it complemented from there on (fl: ket side, bfl: bra
  // side); every later tensor on the wire reads that index complemented
  std::vector<int> fl(n, 0), bfl(n, 0);
  auto leaf = [&](int kind, int gate, int conj, int bit, std::vector<int> idx, int flip = 0) {
    Leaf L;
    L.kind = kind;
    L.gate = gate;
    L.conj = conj;
    L.bit = bit;
    L.flip = flip;
    L.idx = std::move(idx);
    N.leaves.push_back(std::move(L));
  };
  for (int q = 0; q < n; q++)
    if (inq[q]) {
      w[q] = next++;
      leaf(LEAF_KET0, -1, 0, 0, {w[q]});
      N.qubits_kept++;
    }
  // diagonal reduction: a diagonal gate leaves its wires' indices unchanged
  // (they become hyperedges), CNOT keeps its control wire's index
  auto diag = [&](int kind) { return hyper && (kind == TDQ_Z || kind == TDQ_RZ || kind == TDQ_CZ || kind == TDQ_RZZ); };
  // anti-diagonal reduction: X = complement, Y = complement after the phases
  // (i, -i) of its input value (Y[o][i] = [o == 1 - i] Y[1 - i][i])
  auto anti = [&](int kind) { return hyper && (kind == TDQ_X || kind == TDQ_Y); };
  for (int g : kept) {
    const GateRec& G = c->gates[g];
    const int q0 = G.q[0], q1 = G.q[1];
    if (anti(G.kind)) {
      if (G.kind == TDQ_Y) leaf(LEAF_DIAG, g, 0, 0, {w[q0]}, fl[q0]);
      fl[q0] ^= 1;
    } else if (diag(G.kind)) {
      if (gate_arity(G.kind) == 1) leaf(LEAF_DIAG, g, 0, 0, {w[q0]}, fl[q0]);
      else leaf(LEAF_DIAG, g, 0, 0, {w[q0], w[q1]}, fl[q0] | fl[q1] << 1);
    } else if (hyper && G.kind == TDQ_CNOT) {
      const int ob = next++;
      leaf(LEAF_CTRL, g, 0, 0, {w[q0], ob, w[q1]}, fl[q0] | fl[q1] << 2);
      w[q1] = ob;
      fl[q1] = 0;
    } else if (gate_arity(G.kind) == 1) {
      const int o = next++;
      leaf(LEAF_GATE, g, 0, 0, {o, w[q0]}, fl[q0] << 1);
      w[q0] = o;
      fl[q0] = 0;
    } else if (split) {
      // G = sum_s |s><s| (x) V_s: two rank-3 halves joined by a bond
      const int bond = next++, oa = next++, ob = next++;
      leaf(LEAF_HALF0, g, 0, 0, {bond, oa, w[q0]}, fl[q0] << 2);
      leaf(LEAF_HALF1, g, 0, 0, {bond, ob, w[q1]}, fl[q1] << 2);
      w[q0] = oa;
      w[q1] = ob;
      fl[q0] = fl[q1] = 0;
    } else {
      const int oa = next++, ob = next++;
      leaf(LEAF_GATE, g, 0, 0, {oa, ob, w[q0], w[q1]}, fl[q0] << 2 | fl[q1] << 3);
      w[q0] = oa;
      w[q1] = ob;
      fl[q0] = fl[q1] = 0;
    }
  }
  N.gates_kept = (int)kept.size();
  if (output == TDQ_OUT_AMPLITUDE) {
    const std::vector<uint8_t>& bits = c->amps[which];
    for (int q = 0; q < n; q++) leaf(LEAF_BIT, -1, 0, bits[q], {w[q]}, fl[q]);
  } else {
    // observable between the ket legs and the conjugate network's legs
    std::vector<int> bw(n, -1);
    const Term& t = c->terms[which];
    std::vector<char> isz(n, 0);
    for (int q : t.zq) isz[q] = 1;
    for (int q = 0; q < n; q++) {
      if (!inq[q]) continue;
      if (isz[q] && hyper) {  // Z is diagonal: one tensor on the wire, the bra leg is the ket leg
        bw[q] = w[q];
        bfl[q] = fl[q];
        leaf(LEAF_DIAG, -1, 0, 0, {w[q]}, fl[q]);
      } else if (isz[q]) {
        bw[q] = next++;
        leaf(LEAF_OBS_Z, -1, 0, 0, {bw[q], w[q]}, fl[q] << 1);
      } else {
        bw[q] = w[q];  // identity: the bra leg is the ket leg
        bfl[q] = fl[q];
      }
    }
    // the conjugate network, last gate first: a tensor's "out" legs are the
    // bra wires already placed (later in the circuit), its "in" legs new
    for (int i = (int)kept.size() - 1; i >= 0; i--) {
      const int g = kept[i];
      const GateRec& G = c->gates[g];
      const int q0 = G.q[0], q1 = G.q[1];
      if (anti(G.kind)) {  // the phases are those of the earlier (input) value
        if (G.kind == TDQ_Y) leaf(LEAF_DIAG, g, 1, 0, {bw[q0]}, bfl[q0] ^ 1);
        bfl[q0] ^= 1;
      } else if (diag(G.kind)) {
        if (gate_arity(G.kind) == 1) leaf(LEAF_DIAG, g, 1, 0, {bw[q0]}, bfl[q0]);
        else leaf(LEAF_DIAG, g, 1, 0, {bw[q0], bw[q1]}, bfl[q0] | bfl[q1] << 1);
      } else if (hyper && G.kind == TDQ_CNOT) {
        const int ib = next++;
        leaf(LEAF_CTRL, g, 1, 0, {bw[q0], bw[q1], ib}, bfl[q0] | bfl[q1] << 1);
        bw[q1] = ib;
        bfl[q1] = 0;
      } else if (gate_arity(G.kind) == 1) {
        const int in = next++;
        leaf(LEAF_GATE, g, 1, 0, {bw[q0], in}, bfl[q0]);
        bw[q0] = in;
        bfl[q0] = 0;
      } else if (split) {
        const int bond = next++, ia = next++, ib = next++;
        leaf(LEAF_HALF0, g, 1, 0, {bond, bw[q0], ia}, bfl[q0] << 1);
        leaf(LEAF_HALF1, g, 1, 0, {bond, bw[q1], ib}, bfl[q1] << 1);
        bw[q0] = ia;
        bw[q1] = ib;
        bfl[q0] = bfl[q1] = 0;
      } else {
        const int ia = next++, ib = next++;
        leaf(LEAF_GATE, g, 1, 0, {bw[q0], bw[q1], ia, ib}, bfl[q0] | bfl[q1] << 1);
        bw[q0] = ia;
        bw[q1] = ib;
        bfl[q0] = bfl[q1] = 0;
      }
    }
    for (int q = 0; q < n; q++)
      if (inq[q]) leaf(LEAF_BIT, -1, 1, 0, {bw[q]}, bfl[q]);
  }
  N.n_indices = next;
  return 0;
}

std::vector<int> live_counts(const Network& net) {
  std::vector<int> live(net.n_indices, 0);
  for (const Leaf& L : net.leaves)
    for (int i : L.idx) live[i]++;
  for (int& c : live)
    if (c == 1) c = 2;  // an open index: one virtual holder that is never contracted
  return live;
}

std::vector<int> merge_live(const std::vector<int>& a, const std::vector<int>& b, const std::vector<int>& live,
                            int* n_summed) {
  std::vector<int> r;
  int k = 0;
  for (int i : a) {
    const bool on_b = std::find(b.begin(), b.end(), i) != b.end();
    if (!on_b || live[i] > 2) r.push_back(i);
    else k++;
  }
  for (int i : b)
    if (std::find(a.begin(), a.end(), i) == a.end()) r.push_back(i);
  if (n_summed) *n_summed = k;
  return r;
}

// live counts after a and b were contracted into r
static void apply_merge(const std::vector<int>& a, const std::vector<int>& b, const std::vector<int>& r,
                        std::vector<int>& live) {
  for (int i : a) live[i]--;
  for (int i : b) live[i]--;
  for (int i : r) live[i]++;
}

std::vector<std::vector<int>> ssa_indices(const Network& net, const std::vector<Step>& steps,
                                          const std::vector<int>& sliced, std::vector<int>* summed) {
  std::vector<std::vector<int>> T;
  std::vector<char> cut(net.n_indices, 0);
  for (int s : sliced) cut[s] = 1;
  for (const Leaf& L : net.leaves) {
    std::vector<int> v;
    for (int i : L.idx)
      if (!cut[i]) v.push_back(i);
    T.push_back(v);
  }
  std::vector<int> live = live_counts(net);
  if (summed) summed->clear();
  for (const Step& s : steps) {
    int k = 0;
    std::vector<int> r = merge_live(T[s.a], T[s.b], live, &k);
    apply_merge(T[s.a], T[s.b], r, live);
    T.push_back(std::move(r));
    if (summed) summed->push_back(k);
  }
  return T;
}

static double log2_add(double a, double b) {
  if (a < b) std::swap(a, b);
  if (b == -INFINITY) return a;
  return a + std::log2(1.0 + std::exp2(b - a));
}

void plan_measure(Plan& p) {
  std::vector<int> summed;
  auto T = ssa_indices(*p.net, p.steps, p.sliced, &summed);
  const int nl = (int)p.net->leaves.size();
  double lf = -INFINITY, lb = -INFINITY;
  int w = 0;
  for (auto& t : T) w = std::max(w, (int)t.size());
  for (size_t si = 0; si < p.steps.size(); si++) {
    const Step& s = p.steps[si];
    const int r = (int)T[nl + si].size();
    // FLOPs = p (2q - 1), p = 2^|result|, q = 2^|summed| (Sec. 3.2.2, Eq. 5)
    lf = log2_add(lf, (double)r + std::log2(2.0 * std::ldexp(1.0, summed[si]) - 1.0));
    // bytes moved by a step: both operands read, result written (complex64)
    lb = log2_add(lb, std::log2(8.0) + std::log2(std::exp2((double)T[s.a].size()) +
                                                 std::exp2((double)T[s.b].size()) + std::exp2((double)r)));
  }
  p.log2_flops = p.steps.empty() ? 0 : lf;
  p.flops = p.steps.empty() ? 0 : std::exp2(lf + (double)p.sliced.size());
  p.max_log2_width = w;
  p.log2_bytes = p.steps.empty() ? 0 : lb;
}


// Candidate pair.  Ranked by the size heuristic of the greedy pathfinders
// the paper's default finder draws on -- entries of the result minus entries
// of the two operands -- then by FLOPs p(2q-1) (Sec. 3.2.2, Eq. 5), the
// result size and the tensor ids.
struct Cand {
  double cost, flops;
  int rank, i, j;
  bool operator>(const Cand& o) const {
    if (cost != o.cost) return cost > o.cost;
    if (flops != o.flops) return flops > o.flops;
    if (rank != o.rank) return rank > o.rank;
    if (i != o.i) return i > o.i;
    return j > o.j;
  }
};

// Greedy (temperature 0) or Boltzmann random-greedy pairwise path over the
// tensors T0 (index sets; ids < T0.size() are these, id T0.size() + s is the
// result of step s).
std::vector<Step> greedy_path_sets(const std::vector<std::vector<int>>& T0, const std::vector<int>& live0,
                                   double temperature, uint64_t seed) {
  const int nl = (int)T0.size();
  std::vector<std::vector<int>> T = T0;
  std::vector<int> live = live0;
  std::vector<char> alive(nl, 1);
  std::vector<std::vector<int>> holders(live.size());
  for (int t = 0; t < nl; t++)
    for (int i : T[t]) holders[i].push_back(t);
  std::priority_queue<Cand, std::vector<Cand>, std::greater<Cand>> pq;
  std::set<std::pair<int, int>> seen;
  // (costs use the live counts of the moment they are queued; with hyperedges
  // a queued pair's result can shrink later, which the greedy does not revisit)
  auto push = [&](int a, int b) {
    if (a > b) std::swap(a, b);
    if (!seen.insert({a, b}).second) return;
    int k = 0;
    const int r = (int)merge_live(T[a], T[b], live, &k).size();
    const double f = (double)r + std::log2(2.0 * std::ldexp(1.0, k) - 1.0);
    const double c = std::ldexp(1.0, r) - std::ldexp(1.0, (int)T[a].size()) - std::ldexp(1.0, (int)T[b].size());
    pq.push({c, f, r, a, b});
  };
  for (size_t i = 0; i < holders.size(); i++)
    for (size_t u = 0; u < holders[i].size(); u++)
      for (size_t v = u + 1; v < holders[i].size(); v++) push(holders[i][u], holders[i][v]);
  Rng rng(seed);
  std::vector<Step> steps;
  int nlive = nl;
  while (nlive > 1) {
    Cand pick{0, 0, 0, -1, -1};
    if (temperature <= 0) {
      while (!pq.empty()) {
        Cand c = pq.top();
        pq.pop();
        if (alive[c.i] && alive[c.j]) {
          pick = c;
          break;
        }
      }
    } else {
      // sample among the best few live candidates with weights exp(-dcost/T)
      std::vector<Cand> top;
      while (!pq.empty() && top.size() < 8) {
        Cand c = pq.top();
        pq.pop();
        if (alive[c.i] && alive[c.j]) top.push_back(c);
      }
      if (!top.empty()) {
        std::vector<double> wts;
        double tot = 0;
        const double scale = std::max(1.0, std::fabs(top[0].cost));
        for (const Cand& c : top) {
          wts.push_back(std::exp(-(c.cost - top[0].cost) / (temperature * scale)));
          tot += wts.back();
        }
        double u = rng.uniform() * tot;
        size_t k = 0;
        for (; k + 1 < top.size(); k++) {
          if (u < wts[k]) break;
          u -= wts[k];
        }
        pick = top[k];
        for (size_t m = 0; m < top.size(); m++)
          if (m != k) pq.push(top[m]);
      }
    }
    if (pick.i < 0) {  // disconnected: outer product of the two smallest live tensors
      int a = -1, b = -1;
      for (int t = 0; t < (int)T.size(); t++) {
        if (!alive[t]) continue;
        if (a < 0 || T[t].size() < T[a].size()) { b = a; a = t; }
        else if (b < 0 || T[t].size() < T[b].size()) b = t;
      }
      pick = {0, 0, 0, std::min(a, b), std::max(a, b)};
    }
    const int id = (int)T.size();
    std::vector<int> r = merge_live(T[pick.i], T[pick.j], live, nullptr);
    apply_merge(T[pick.i], T[pick.j], r, live);
    for (int x : {pick.i, pick.j})
      for (int i : T[x]) {
        auto& h = holders[i];
        h.erase(std::remove_if(h.begin(), h.end(), [&](int y) { return y == pick.i || y == pick.j; }), h.end());
      }
    T.push_back(std::move(r));
    alive.push_back(1);
    alive[pick.i] = alive[pick.j] = 0;
    steps.push_back({pick.i, pick.j});
    nlive--;
    for (int i : T[id]) {
      auto& h = holders[i];
      for (int x : h)
        if (alive[x]) push(id, x);
      h.push_back(id);
    }
  }
  return steps;
}

static std::vector<Step> greedy_path(const Network& net, double temperature, uint64_t seed) {
  std::vector<std::vector<int>> T0;
  for (const Leaf& L : net.leaves) T0.push_back(L.idx);
  return greedy_path_sets(T0, live_counts(net), temperature, seed);
}

// Rank simplification (Sec. 3.2.1, the local processing before the path
// search): while two live tensors share an index and contracting them gives
// a tensor with no more indices than the larger of the two, contract the pair
// whose result has the fewest indices (then the one that removes the most,
// then the lowest ids).  The contractions never widen the network; they
// become the first steps of every path, and the path finders work on what is
// left.  Returns those steps (SSA over the network's leaves); `rest` receives
// the SSA ids of the tensors left, in increasing order.
std::vector<Step> rank_simplify(const Network& net, std::vector<int>& rest) {
  const int nl = (int)net.leaves.size();
  std::vector<std::vector<int>> T;
  for (const Leaf& L : net.leaves) T.push_back(L.idx);
  std::vector<int> live = live_counts(net);
  std::vector<std::vector<int>> holders(net.n_indices);
  for (int t = 0; t < nl; t++)
    for (int i : T[t]) holders[i].push_back(t);
  std::vector<char> alive(nl, 1);
  std::vector<Step> steps;
  for (;;) {
    int ba = -1, bb = -1, br = 0, bgain = 0;
    std::vector<int> bres;
    for (int a = 0; a < (int)T.size(); a++) {
      if (!alive[a]) continue;
      for (int i : T[a])
        for (int b : holders[i]) {
          if (b <= a || !alive[b]) continue;
          std::vector<int> r = merge_live(T[a], T[b], live, nullptr);
          const int mx = (int)std::max(T[a].size(), T[b].size());
          if ((int)r.size() > mx) continue;
          const int gain = mx - (int)r.size();
          const bool better = ba < 0 || (int)r.size() < br || ((int)r.size() == br && gain > bgain);
          if (better) {
            ba = a, bb = b, br = (int)r.size(), bgain = gain;
            bres = std::move(r);
          }
        }
    }
    if (ba < 0) break;
    apply_merge(T[ba], T[bb], bres, live);
    alive[ba] = alive[bb] = 0;
    const int id = (int)T.size();
    for (int i : bres) holders[i].push_back(id);
    T.push_back(bres);
    alive.push_back(1);
    steps.push_back({ba, bb});
  }
  rest.clear();
  for (int t = 0; t < (int)T.size(); t++)
    if (alive[t]) rest.push_back(t);
  return steps;
}

// The path of `method` (greedy with the given temperature, or the partition
// tree) after rank simplification: the simplification's steps, then the
// finder's path over the tensors left, mapped back to SSA ids.
static std::vector<Step> simplified_path(const Network& net, bool partition, double temperature, uint64_t seed) {
  std::vector<int> rest;
  std::vector<Step> steps = rank_simplify(net, rest);
  if (rest.size() <= 1) return steps;
  // the tensors left as a network of their own (the finders read only the
  // index sets)
  Network sub;
  sub.n_indices = net.n_indices;
  auto T = ssa_indices(net, steps, {});
  for (int id : rest) {
    Leaf L;
    L.idx = T[id];
    sub.leaves.push_back(L);
  }
  const std::vector<Step> tail = partition ? partition_tree(sub, seed) : greedy_path(sub, temperature, seed);
  const int nl = (int)net.leaves.size(), nr = (int)rest.size(), n0 = (int)steps.size();
  auto gid = [&](int x) { return x < nr ? rest[x] : nl + n0 + (x - nr); };
  for (const Step& st : tail) steps.push_back({gid(st.a), gid(st.b)});
  return steps;
}

// Greedy slicing (Sec. 3.2.3): while some tensor is wider than the target,
// pick the index with the largest summed log2 size over the oversize tensors
// that contain it (ties at random) and slice it.
static std::vector<int> greedy_slices(const Network& net, const std::vector<Step>& steps,
                                      int target, uint64_t seed) {
  std::vector<int> sliced;
  Rng rng(seed ^ 0x51ced51ced51ceull);
  if (target <= 0) return sliced;
  for (int round = 0; round < 64; round++) {
    auto T = ssa_indices(net, steps, sliced);
    std::vector<double> score(net.n_indices, 0.0);
    bool over = false;
    for (const auto& t : T) {
      if ((int)t.size() <= target) continue;
      over = true;
      for (int i : t) score[i] += (double)t.size();
    }
    if (!over) break;
    double best = 0;
    for (double s : score) best = std::max(best, s);
    std::vector<int> ties;
    for (int i = 0; i < net.n_indices; i++)
      if (score[i] == best && best > 0) ties.push_back(i);
    if (ties.empty()) break;
    sliced.push_back(ties[rng.next() % ties.size()]);
  }
  return sliced;
}

}  // namespace tdq

using namespace tdq;

extern "C" {

tdq_status tdq_network_build(const tdq_circuit* c, const tdq_net_opts* o, tdq_network** out) {
  if (!c || !o || !out) return fail(TDQ_ERR_ARG, "tdq_network_build: NULL argument");
  *out = nullptr;
  if (o->output == TDQ_OUT_EXPVAL) {
    if (o->index < 0 || o->index >= (int)c->terms.size())
      return fail(TDQ_ERR_ARG, "tdq_network_build: no such observable term");
  } else if (o->output == TDQ_OUT_AMPLITUDE) {
    if (o->index < 0 || o->index >= (int)c->amps.size())
      return fail(TDQ_ERR_ARG, "tdq_network_build: no such amplitude request");
  } else {
    return fail(TDQ_ERR_ARG, "tdq_network_build: bad output kind");
  }
  auto net = std::make_shared<Network>();
  build_network(c, o->output, o->index, o->lightcone, o->split_2q, o->hyper, *net);
  tdq_network* h = new (std::nothrow) tdq_network();
  if (!h) return fail(TDQ_ERR_OOM, "tdq_network_build: host allocation");
  h->net = net;
  *out = h;
  return ok();
}

tdq_status tdq_network_info(const tdq_network* h, int* n_tensors, int* n_indices, int* n_qubits,
                            int* n_gates) {
  if (!h) return fail(TDQ_ERR_ARG, "tdq_network_info: NULL network");
  if (n_tensors) *n_tensors = (int)h->net->leaves.size();
  if (n_indices) *n_indices = h->net->n_indices;
  if (n_qubits) *n_qubits = h->net->qubits_kept;
  if (n_gates) *n_gates = h->net->gates_kept;
  return ok();
}

tdq_status tdq_network_tensor(const tdq_network* h, int i, int* kind, int* gate, int* conj,
                              int* bit, int* rank, int* idx) {
  if (!h || i < 0 || i >= (int)h->net->leaves.size())
    return fail(TDQ_ERR_ARG, "tdq_network_tensor: bad tensor");
  const Leaf& L = h->net->leaves[i];
  if (kind) *kind = L.kind;
  if (gate) *gate = L.gate;
  if (conj) *conj = L.conj;
  if (bit) *bit = L.bit;
  if (rank) *rank = (int)L.idx.size();
  if (idx)
    for (size_t k = 0; k < L.idx.size(); k++) idx[k] = L.idx[k];
  return ok();
}

tdq_status tdq_network_tensor_flips(const tdq_network* h, int i, int* flip) {
  if (!h || !flip || i < 0 || i >= (int)h->net->leaves.size())
    return fail(TDQ_ERR_ARG, "tdq_network_tensor_flips: bad tensor");
  *flip = h->net->leaves[i].flip;
  return ok();
}

tdq_status tdq_network_destroy(tdq_network* h) {
  delete h;
  return ok();
}

tdq_status tdq_plan_find(const tdq_network* h, const tdq_plan_opts* o, tdq_plan** out) {
  if (!h || !o || !out) return fail(TDQ_ERR_ARG, "tdq_plan_find: NULL argument");
  *out = nullptr;
  if (o->method != TDQ_PATH_GREEDY && o->method != TDQ_PATH_RANDOM_GREEDY && o->method != TDQ_PATH_PARTITION)
    return fail(TDQ_ERR_ARG, "tdq_plan_find: method must be greedy, random-greedy or partition");
  if (o->target_log2 < 0 || o->target_log2 > 40) return fail(TDQ_ERR_ARG, "tdq_plan_find: bad target");
  if (o->slice_trials < 0 || o->slice_trials > (1 << 20) || o->slice_final < 0 || o->slice_final > (1 << 20))
    return fail(TDQ_ERR_ARG, "tdq_plan_find: slice_trials and slice_final must be in [0, 2^20]");
  if (o->rank_simplify != 0 && o->rank_simplify != 1)
    return fail(TDQ_ERR_ARG, "tdq_plan_find: rank_simplify must be 0 or 1");
  tdq_plan* p = new (std::nothrow) tdq_plan();
  if (!p) return fail(TDQ_ERR_OOM, "tdq_plan_find: host allocation");
  p->plan.net = h->net;
  const Network& net = *h->net;
  const double temp = o->method == TDQ_PATH_GREEDY ? 0.0 : (o->temperature > 0 ? o->temperature : 1.0);
  const int trials = o->method == TDQ_PATH_GREEDY ? 1 : std::max(1, o->repeats);
  // phase 1: candidate trees, each with its own slicing (the single greedy
  // rule, or the best of slice_trials randomised slicings)
  std::vector<Plan> cand(trials);
  std::atomic<bool> oom{false};  // set by any trial thread
  auto one = [&](int r) {
    try {
      Plan& c = cand[r];
      c.net = h->net;
      const uint64_t seed = o->seed + (uint64_t)r;
      if (o->rank_simplify)
        c.steps = simplified_path(net, o->method == TDQ_PATH_PARTITION, temp, seed);
      else
        c.steps = o->method == TDQ_PATH_PARTITION ? partition_tree(net, seed) : greedy_path(net, temp, seed);
      // the single greedy slicing competes in phase 1, so the two-phase
      // search never ends above it
      c.sliced = greedy_slices(net, c.steps, o->target_log2, seed);
      if (o->slice_trials > 0)
        c.sliced = best_slices(net, c.steps, o->target_log2, o->slice_trials, seed, &c.sliced, false);
      plan_measure(c);
    } catch (...) {  // allocation failure in a trial (no exception leaves the C ABI)
      oom = true;
    }
  };
  if (trials > 1) {
    parallel_trials(trials, one);
  } else {
    one(0);
  }
  if (oom) {
    delete p;
    return fail(TDQ_ERR_OOM, "tdq_plan_find: host allocation");
  }
  int best = 0;
  for (int r = 1; r < trials; r++)
    if (cand[r].flops < cand[best].flops) best = r;
  p->plan = cand[best];
  // phase 2: more slicing trials on the winning tree
  if (o->slice_final > 0 && o->target_log2 > 0) {
    try {
      p->plan.sliced = best_slices(net, p->plan.steps, o->target_log2, o->slice_final, o->seed ^ 0xf1a1ull,
                                   &p->plan.sliced, true);
    } catch (...) {
      delete p;
      return fail(TDQ_ERR_OOM, "tdq_plan_find: host allocation");
    }
    plan_measure(p->plan);
  }
  *out = p;
  return ok();
}

tdq_status tdq_plan_from_path(const tdq_network* h, const int* pairs, int n_steps,
                              const int* sliced, int n_sliced, tdq_plan** out) {
  if (!h || !out || (n_steps > 0 && !pairs) || (n_sliced > 0 && !sliced))
    return fail(TDQ_ERR_ARG, "tdq_plan_from_path: NULL argument");
  *out = nullptr;
  const int nl = (int)h->net->leaves.size();
  if (n_steps != nl - 1) return fail(TDQ_ERR_ARG, "tdq_plan_from_path: need n_tensors - 1 steps");
  std::vector<char> used(2 * nl, 0);
  std::vector<Step> steps;
  for (int s = 0; s < n_steps; s++) {
    const int a = pairs[2 * s], b = pairs[2 * s + 1];
    const int lim = nl + s;
    if (a < 0 || b < 0 || a >= lim || b >= lim || a == b || used[a] || used[b])
      return fail(TDQ_ERR_ARG, "tdq_plan_from_path: invalid or reused tensor id at step " + std::to_string(s));
    used[a] = used[b] = 1;
    steps.push_back({a, b});
  }
  std::vector<int> sl;
  for (int i = 0; i < n_sliced; i++) {
    if (sliced[i] < 0 || sliced[i] >= h->net->n_indices)
      return fail(TDQ_ERR_ARG, "tdq_plan_from_path: bad sliced index");
    sl.push_back(sliced[i]);
  }
  tdq_plan* p = new (std::nothrow) tdq_plan();
  if (!p) return fail(TDQ_ERR_OOM, "tdq_plan_from_path: host allocation");
  p->plan.net = h->net;
  p->plan.steps = steps;
  p->plan.sliced = sl;
  plan_measure(p->plan);
  *out = p;
  return ok();
}

tdq_status tdq_plan_stats(const tdq_plan* p, tdq_stats* s) {
  if (!p || !s) return fail(TDQ_ERR_ARG, "tdq_plan_stats: NULL argument");
  s->log2_flops_per_slice = p->plan.log2_flops;
  s->flops = p->plan.flops;
  s->max_log2_width = p->plan.max_log2_width;
  s->n_sliced = (int)p->plan.sliced.size();
  s->n_steps = (int)p->plan.steps.size();
  s->log2_bytes_per_slice = p->plan.log2_bytes;
  return ok();
}

tdq_status tdq_plan_path(const tdq_plan* p, int* pairs, int* sliced) {
  if (!p) return fail(TDQ_ERR_ARG, "tdq_plan_path: NULL plan");
  if (pairs)
    for (size_t s = 0; s < p->plan.steps.size(); s++) {
      pairs[2 * s] = p->plan.steps[s].a;
      pairs[2 * s + 1] = p->plan.steps[s].b;
    }
  if (sliced)
    for (size_t i = 0; i < p->plan.sliced.size(); i++) sliced[i] = p->plan.sliced[i];
  return ok();
}

tdq_status tdq_plan_destroy(tdq_plan* p) {
  delete p;
  return ok();
}

}  // extern "C"
