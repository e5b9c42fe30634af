// Contraction trees by recursive bipartition of the network's hypergraph
// (Sec. 3.2.2, the hypergraph-based pathfinder) and the two-phase,
// slicing-aware choice of tree and sliced indices (Sec. 3.2.3).
//
// Tensors are the vertices of the hypergraph and indices its edges.  A tree
// is built top-down: the node holding the tensor set S is split into children
// A and B that minimise
//     cut(A, B) + w * |outer(A) - outer(B)|,
// where cut counts the indices with tensors on both sides (each one doubles q
// in the cost p(2q - 1) of contracting A with B, Eq. 5) and outer(X) counts
// the indices X shares with anything outside X, i.e. the rank of X's
// intermediate tensor: spreading S's outer indices evenly over the children
// lowers p in the children's own contractions and the memory m q + n q of
// the contraction at S.  Each side holds at most (1 + eps) |S| / 2 tensors.
// Sets of at most `cutoff` tensors are finished by the greedy pathfinder.  The
// pairwise path is the tree read bottom-up.
//
// The bipartitioner is multilevel, as KaHyPar (which the paper uses here) is:
// the node's hypergraph is coarsened by heavy-edge matching, the coarsest
// graph is split from breadth-first-grown starting halves, and each level on
// the way back is refined by Fiduccia-Mattheyses passes (one vertex moved at
// a time, best gain first, each vertex once per pass, rolled back to the
// best prefix).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <exception>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>

#include "network.h"

namespace tdq {

namespace {

struct TreeParams {
  double eps;  // imbalance: each side holds at most (1 + eps) |S| / 2 tensors
  double w;    // weight of |outer(A) - outer(B)| against the cut
  int cutoff;  // sets of at most this many tensors finish with greedy
  int starts;  // starting halves refined per bisection
};

// Hypergraph of one tree node: vertices are clusters of the node's tensors
// (weight = tensors), edges are indices (weight = parallel indices merged),
// `outer` marks an edge that also reaches tensors outside the node.
struct HG {
  std::vector<int> vw, ew;
  std::vector<std::vector<int>> pins, vedges;
  std::vector<char> outer;
  int nv() const { return (int)vw.size(); }
  int total() const {
    int t = 0;
    for (int w : vw) t += w;
    return t;
  }
  void index() {
    vedges.assign(vw.size(), {});
    for (size_t e = 0; e < pins.size(); e++)
      for (int v : pins[e]) vedges[v].push_back((int)e);
  }
};

// Two-way partition state of an HG with the objective cut + w |D|,
// D = outer(side 0) - outer(side 1), counted with edge weights.
class Bipart {
 public:
  Bipart(const HG& g, double w, int maxside) : g_(g), w_(w), maxside_(maxside) {}

  std::vector<char> side;

  void recount() {
    cnt_.assign(2 * g_.pins.size(), 0);
    size_[0] = size_[1] = 0;
    for (int v = 0; v < g_.nv(); v++) size_[(int)side[v]] += g_.vw[v];
    cut_ = 0;
    D_ = 0;
    for (size_t e = 0; e < g_.pins.size(); e++) {
      for (int v : g_.pins[e]) cnt_[2 * e + side[v]]++;
      const int c0 = cnt_[2 * e], c1 = cnt_[2 * e + 1], w = g_.ew[e];
      const bool out = g_.outer[e];
      cut_ += w * (c0 > 0 && c1 > 0);
      D_ += w * ((int)(c0 > 0 && (c1 > 0 || out)) - (int)(c1 > 0 && (c0 > 0 || out)));
    }
  }

  double cost() const { return cut_ + w_ * std::abs(D_); }
  int size(int s) const { return size_[s]; }

  // Fiduccia-Mattheyses passes: the unlocked vertex with the best gain (ties:
  // from the heavier side) moves, if the other side stays within maxside;
  // each pass is rolled back to its best prefix.
  void refine() {
    const int n = g_.nv();
    std::vector<int> gcut(n), gD(n);
    std::vector<char> locked(n);
    std::vector<int> moved;
    for (int pass = 0; pass < 16; pass++) {
      for (int v = 0; v < n; v++) delta(v, &gcut[v], &gD[v]);
      std::fill(locked.begin(), locked.end(), 0);
      moved.clear();
      double best = cost();
      size_t best_len = 0;
      const size_t patience = (size_t)std::max(50, n / 4);
      for (int m = 0; m < n; m++) {
        int pick = -1;
        double pg = 0;
        bool plarge = false;
        for (int v = 0; v < n; v++) {
          const int s = side[v];
          if (locked[v] || size_[1 - s] + g_.vw[v] > maxside_) continue;
          const double g = -(gcut[v] + w_ * (std::abs(D_ + gD[v]) - std::abs(D_)));
          const bool large = size_[s] > size_[1 - s];
          if (pick < 0 || g > pg + 1e-9 || (g > pg - 1e-9 && large && !plarge)) {
            pick = v;
            pg = g;
            plarge = large;
          }
        }
        if (pick < 0) break;
        move(pick);
        locked[pick] = 1;
        moved.push_back(pick);
        for (int e : g_.vedges[pick])
          for (int u : g_.pins[e])
            if (!locked[u]) delta(u, &gcut[u], &gD[u]);
        const double c = cost();
        if (c < best - 1e-9) {
          best = c;
          best_len = moved.size();
        } else if (moved.size() - best_len > patience) {
          break;
        }
      }
      for (size_t k = moved.size(); k > best_len; k--) move(moved[k - 1]);
      if (best_len == 0) break;
    }
  }

 private:
  // change of the cut and of D if vertex v changes side
  void delta(int v, int* dcut, int* dD) const {
    const int s = side[v], t = 1 - s;
    int dc = 0, ds = 0, dt = 0;
    for (int e : g_.vedges[v]) {
      const int cs = cnt_[2 * e + s], ct = cnt_[2 * e + t], w = g_.ew[e];
      const bool out = g_.outer[e];
      dc += w * ((int)(cs > 1) - (int)(cs > 0 && ct > 0));
      ds += w * ((int)(cs > 1) - (int)(cs > 0 && (ct > 0 || out)));
      dt += w * ((int)(cs > 1 || out) - (int)(ct > 0 && (cs > 0 || out)));
    }
    *dcut = dc;
    *dD = s == 0 ? ds - dt : dt - ds;
  }

  void move(int v) {
    int dc, dD;
    delta(v, &dc, &dD);
    const int s = side[v];
    for (int e : g_.vedges[v]) {
      cnt_[2 * e + s]--;
      cnt_[2 * e + 1 - s]++;
    }
    size_[s] -= g_.vw[v];
    size_[1 - s] += g_.vw[v];
    side[v] = (char)(1 - s);
    cut_ += dc;
    D_ += dD;
  }

  const HG& g_;
  const double w_;
  const int maxside_;
  std::vector<int> cnt_;
  int size_[2] = {0, 0};
  int cut_ = 0, D_ = 0;
};

// One coarsening step: every vertex, in random order, joins the unmatched
// neighbour with the highest rating sum_e w(e) / (|e| - 1) / (w(u) w(v))
// (heavy edges first, light vertices first) unless the pair would outweigh
// maxw; parallel edges merge and edges inside one cluster vanish.
static bool coarsen(const HG& g, int maxw, Rng& rng, HG& c, std::vector<int>& map) {
  const int n = g.nv();
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  for (int i = n - 1; i > 0; i--) std::swap(order[i], order[(int)(rng.next() % (uint64_t)(i + 1))]);
  map.assign(n, -1);
  std::vector<double> rating(n, 0.0);
  std::vector<int> touched;
  int nc = 0;
  c.vw.clear();
  for (int v : order) {
    if (map[v] >= 0) continue;
    touched.clear();
    for (int e : g.vedges[v]) {
      if (g.pins[e].size() < 2) continue;
      const double r = (double)g.ew[e] / (double)(g.pins[e].size() - 1);
      for (int u : g.pins[e])
        if (u != v && map[u] < 0 && g.vw[u] + g.vw[v] <= maxw) {
          if (rating[u] == 0) touched.push_back(u);
          rating[u] += r;
        }
    }
    int best = -1;
    double br = 0;
    for (int u : touched) {
      const double r = rating[u] / ((double)g.vw[u] * (double)g.vw[v]);
      if (r > br) {
        br = r;
        best = u;
      }
      rating[u] = 0;
    }
    map[v] = nc;
    int w = g.vw[v];
    if (best >= 0) {
      map[best] = nc;
      w += g.vw[best];
    }
    c.vw.push_back(w);
    nc++;
  }
  if (nc > n * 9 / 10) return false;  // stalled
  c.pins.clear();
  c.ew.clear();
  c.outer.clear();
  std::map<std::pair<std::vector<int>, char>, int> seen;
  for (size_t e = 0; e < g.pins.size(); e++) {
    std::vector<int> p;
    for (int v : g.pins[e]) p.push_back(map[v]);
    std::sort(p.begin(), p.end());
    p.erase(std::unique(p.begin(), p.end()), p.end());
    if (p.size() < 2 && !g.outer[e]) continue;
    auto key = std::make_pair(p, g.outer[e]);
    auto it = seen.find(key);
    if (it != seen.end()) {
      c.ew[it->second] += g.ew[e];
      continue;
    }
    seen.emplace(key, (int)c.pins.size());
    c.pins.push_back(p);
    c.ew.push_back(g.ew[e]);
    c.outer.push_back(g.outer[e]);
  }
  c.index();
  return true;
}

class TreeBuilder {
 public:
  explicit TreeBuilder(const Network& net)
      : net_(net), nl_((int)net.leaves.size()), holders_(net.n_indices), emark_(net.n_indices, -1),
        live_(live_counts(net)) {
    for (int t = 0; t < nl_; t++)
      for (int i : net.leaves[t].idx) holders_[i].push_back(t);
  }

  std::vector<Step> build(const TreeParams& P, Rng& rng) {
    P_ = P;
    rng_ = &rng;
    steps_.clear();
    std::vector<int> all(nl_);
    std::iota(all.begin(), all.end(), 0);
    if (nl_ > 1) node(all);
    return steps_;
  }

 private:
  // SSA id of the tensor that contracting the leaves S produces
  int node(const std::vector<int>& S) {
    if (S.size() == 1) return S[0];
    if ((int)S.size() <= P_.cutoff) {
      std::vector<std::vector<int>> T0;
      for (int s : S) T0.push_back(net_.leaves[s].idx);
      std::vector<int> id = S;
      for (const Step& st : greedy_path_sets(T0, live_, 0.0, 0)) {
        steps_.push_back({id[st.a], id[st.b]});
        id.push_back(nl_ + (int)steps_.size() - 1);
      }
      return id.back();
    }
    std::vector<char> side;
    bisect(S, side);
    std::vector<int> A, B;
    for (size_t k = 0; k < S.size(); k++) (side[k] ? B : A).push_back(S[k]);
    const int ra = node(A), rb = node(B);
    steps_.push_back({ra, rb});
    return nl_ + (int)steps_.size() - 1;
  }

  // hypergraph of the leaves S: vertex k is S[k]
  HG local_graph(const std::vector<int>& S) {
    HG g;
    const int n = (int)S.size();
    g.vw.assign(n, 1);
    std::vector<int> touched;
    for (int k = 0; k < n; k++)
      for (int i : net_.leaves[S[k]].idx) {
        if (emark_[i] < 0) {
          emark_[i] = (int)g.pins.size();
          g.pins.push_back({});
          touched.push_back(i);
        }
        g.pins[emark_[i]].push_back(k);
      }
    for (int i : touched) {
      const size_t np = g.pins[emark_[i]].size();
      // outer: a tensor outside S holds the index, or it is an open index of
      // the whole network
      g.outer.push_back(np < holders_[i].size() || holders_[i].size() == 1);
      g.ew.push_back(1);
      emark_[i] = -1;
    }
    g.index();
    return g;
  }

  // starting halves grown breadth-first (by weight) from random vertices
  void grow(const HG& g, int maxside, std::vector<char>& side) {
    const int n = g.nv(), half = g.total() / 2;
    side.assign(n, 0);
    std::vector<char> seen(n, 0);
    std::vector<int> queue;
    size_t head = 0;
    int grown = 0, nseen = 0;
    while (grown < half && nseen < n) {
      if (head == queue.size()) {
        int v = (int)(rng_->next() % (uint64_t)n);
        while (seen[v]) v = (v + 1) % n;
        seen[v] = 1;
        nseen++;
        queue.push_back(v);
      }
      const int v = queue[head++];
      if (grown + g.vw[v] > maxside) continue;
      side[v] = 1;
      grown += g.vw[v];
      for (int e : g.vedges[v])
        for (int u : g.pins[e])
          if (!seen[u]) {
            seen[u] = 1;
            nseen++;
            queue.push_back(u);
          }
    }
  }

  // multilevel bisection: coarsen, partition the coarsest graph from several
  // starting halves, then project back level by level with refinement
  void bisect(const std::vector<int>& S, std::vector<char>& out) {
    const int n = (int)S.size();
    const int maxside = std::min(n - 1, std::max((n + 1) / 2, (int)std::floor((1.0 + P_.eps) * n / 2)));
    std::vector<HG> levels;
    std::vector<std::vector<int>> maps;
    levels.push_back(local_graph(S));
    const int maxw = std::max(2, n / 40);
    while (levels.back().nv() > 80) {
      HG c;
      std::vector<int> map;
      if (!coarsen(levels.back(), maxw, *rng_, c, map)) break;
      levels.push_back(std::move(c));
      maps.push_back(std::move(map));
    }
    std::vector<char> side;
    {
      const HG& g = levels.back();
      double best = 0;
      for (int st = 0; st < P_.starts; st++) {
        Bipart bp(g, P_.w, maxside);
        grow(g, maxside, bp.side);
        bp.recount();
        bp.refine();
        if (bp.size(0) == 0 || bp.size(1) == 0) continue;
        if (side.empty() || bp.cost() < best - 1e-9) {
          best = bp.cost();
          side = bp.side;
        }
      }
    }
    if (side.empty()) {  // no balanced start: split by position
      side.assign(levels.back().nv(), 0);
      side[0] = 1;
    }
    for (int l = (int)levels.size() - 2; l >= 0; l--) {
      Bipart bp(levels[l], P_.w, maxside);
      bp.side.resize(levels[l].nv());
      for (int v = 0; v < levels[l].nv(); v++) bp.side[v] = side[maps[l][v]];
      bp.recount();
      bp.refine();
      side = bp.side;
    }
    out = side;
  }

  const Network& net_;
  const int nl_;
  std::vector<std::vector<int>> holders_;
  std::vector<int> emark_;
  std::vector<int> live_;  // holders of every index in the whole network (live_counts)
  TreeParams P_{};
  Rng* rng_ = nullptr;
  std::vector<Step> steps_;
};

// Sliced-path FLOPs without re-deriving index sets: slicing index i removes
// it from every SSA tensor that holds it and from the contracted set of the
// step that sums it, so tensor sizes and per-step contracted counts are
// updated by decrements.
class SliceEval {
 public:
  SliceEval(const Network& net, const std::vector<Step>& steps)
      : steps_(steps), nl_((int)net.leaves.size()), ni_(net.n_indices) {
    T_ = ssa_indices(net, steps, {}, &shared0_);
    holds_.assign(ni_, {});
    for (size_t t = 0; t < T_.size(); t++)
      for (int i : T_[t]) holds_[i].push_back((int)t);
    // the step that sums each index: on both operands, not on the result
    step_of_.assign(ni_, -1);
    for (size_t s = 0; s < steps.size(); s++) {
      const auto& b = T_[steps[s].b];
      const auto& r = T_[nl_ + s];
      for (int i : T_[steps[s].a])
        if (std::find(b.begin(), b.end(), i) != b.end() && std::find(r.begin(), r.end(), i) == r.end())
          step_of_[i] = (int)s;
    }
  }

  // FLOPs of all slices with the indices `sliced` cut
  double flops(const std::vector<int>& sliced) const {
    std::vector<int> sz, sh;
    start(sz, sh);
    for (int i : sliced) cut(i, sz, sh);
    return total(sz, sh, (int)sliced.size());
  }

  // Greedy slicing (Sec. 3.2.3) until no tensor exceeds 2^target entries:
  // every index of the oversize tensors scores the summed log2 sizes of the
  // oversize tensors holding it; tau = 0 slices the best (ties at random),
  // tau > 0 draws with weights exp((score - best) / (tau * best)).
  double trial(int target, double tau, Rng& rng, std::vector<int>& sliced) const {
    std::vector<int> sz, sh;
    start(sz, sh);
    sliced.clear();
    std::vector<char> is_cut(ni_, 0);
    std::vector<double> score(ni_, 0.0);
    std::vector<int> over, touched, ties;
    for (size_t t = 0; t < sz.size(); t++)
      if (sz[t] > target) over.push_back((int)t);
    for (int round = 0; round < 64; round++) {
      over.erase(std::remove_if(over.begin(), over.end(), [&](int t) { return sz[t] <= target; }), over.end());
      if (over.empty()) break;
      touched.clear();
      for (int t : over)
        for (int i : T_[t])
          if (!is_cut[i]) {
            if (score[i] == 0) touched.push_back(i);
            score[i] += sz[t];
          }
      if (touched.empty()) break;
      double best = 0;
      for (int i : touched) best = std::max(best, score[i]);
      int pick = -1;
      if (tau <= 0) {
        ties.clear();
        for (int i : touched)
          if (score[i] == best) ties.push_back(i);
        pick = ties[rng.next() % ties.size()];
      } else {
        double tot = 0;
        for (int i : touched) tot += std::exp((score[i] - best) / (tau * best));
        double u = rng.uniform() * tot;
        for (int i : touched) {
          pick = i;
          u -= std::exp((score[i] - best) / (tau * best));
          if (u < 0) break;
        }
      }
      for (int i : touched) score[i] = 0;
      is_cut[pick] = 1;
      sliced.push_back(pick);
      cut(pick, sz, sh);
    }
    return total(sz, sh, (int)sliced.size());
  }

 private:
  void start(std::vector<int>& sz, std::vector<int>& sh) const {
    sz.resize(T_.size());
    for (size_t t = 0; t < T_.size(); t++) sz[t] = (int)T_[t].size();
    sh = shared0_;
  }
  void cut(int i, std::vector<int>& sz, std::vector<int>& sh) const {
    for (int t : holds_[i]) sz[t]--;
    if (step_of_[i] >= 0) sh[step_of_[i]]--;
  }
  // sum over steps of p (2q - 1), p = 2^|result|, q = 2^|contracted| (Eq. 5), times 2^slices
  double total(const std::vector<int>& sz, const std::vector<int>& sh, int nsl) const {
    double f = 0;
    for (size_t s = 0; s < steps_.size(); s++)
      f += std::ldexp(1.0, sz[nl_ + s]) * (std::ldexp(2.0, sh[s]) - 1.0);
    return std::ldexp(f, nsl);
  }

  const std::vector<Step>& steps_;
  int nl_, ni_;
  std::vector<std::vector<int>> T_, holds_;
  std::vector<int> step_of_, shared0_;
};

// fn(k, worker) for k in [0, n) on up to hardware_concurrency threads; the
// first exception a worker throws is rethrown here after every worker ended
template <class F>
void parallel_for(int n, F&& fn) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::max(1, std::min({n, hw, 32}));
  if (nt == 1) {
    for (int k = 0; k < n; k++) fn(k, 0);
    return;
  }
  std::atomic<int> next{0};
  std::atomic<bool> failed{false};
  std::exception_ptr err;
  std::mutex mu;
  std::vector<std::thread> pool;
  for (int w = 0; w < nt; w++)
    pool.emplace_back([&, w] {
      try {
        for (int k = next++; k < n && !failed; k = next++) fn(k, w);
      } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        if (!err) err = std::current_exception();
        failed = true;
      }
    });
  for (auto& th : pool) th.join();
  if (err) std::rethrow_exception(err);
}

}  // namespace

std::vector<Step> partition_tree(const Network& net, uint64_t seed) {
  Rng rng(seed ^ 0x9a27717104e5ull);
  // per-trial hyper-parameters, drawn like the repeated trials of Sec. 3.2.2
  TreeParams P;
  P.eps = 0.02 + 0.58 * rng.uniform();
  P.w = 0.5 * rng.uniform();
  P.cutoff = 4 + (int)(rng.next() % 21);
  P.starts = 4;
  TreeBuilder tb(net);
  return tb.build(P, rng);
}

std::vector<int> best_slices(const Network& net, const std::vector<Step>& steps, int target, int trials,
                             uint64_t seed, const std::vector<int>* incumbent, bool threads) {
  std::vector<int> best;
  if (target <= 0) return best;
  SliceEval ev(net, steps);
  double fbest = incumbent ? ev.flops(*incumbent) : INFINITY;
  if (incumbent) best = *incumbent;
  std::vector<std::vector<int>> got(trials);
  std::vector<double> f(trials);
  auto one = [&](int k, int) {
    Rng rng(seed * 0x9e3779b97f4a7c15ull + 0x5eed + (uint64_t)k);
    // trial 0 keeps the plain rule; the others draw with a random temperature
    const double tau = k == 0 ? 0.0 : 0.3 * rng.uniform();
    f[k] = ev.trial(target, tau, rng, got[k]);
  };
  if (threads) {
    parallel_for(trials, one);
  } else {
    for (int k = 0; k < trials; k++) one(k, 0);
  }
  for (int k = 0; k < trials; k++)
    if (f[k] < fbest || (f[k] == fbest && got[k].size() < best.size())) {
      fbest = f[k];
      best = got[k];
    }
  return best;
}

void parallel_trials(int n, const std::function<void(int)>& fn) {
  parallel_for(n, [&](int k, int) { fn(k); });
}

}  // namespace tdq
