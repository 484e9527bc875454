// Contraction orderings of Section 3.1: Stoch (Algorithm 2) and LG
// (Algorithm 1), plus the per-step label layout used by the executors.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>

#include "qtc_internal.h"

namespace qtc {

namespace {

// Live tensors of a partially contracted network.  Contracting A and B sums
// every label whose live holders are all among {A, B}; the others stay (a
// label also held elsewhere is a batch index, Eq. 1 with hyperedges).
struct TNState {
  std::vector<std::vector<int>> lab;      // per tensor id, sorted
  std::vector<char> alive;
  std::vector<std::vector<int>> holders;  // per label: live tensor ids
  std::vector<Step> steps;
  int n_live = 0;

  explicit TNState(const Network& net) {
    holders.resize(net.n_labels);
    for (size_t i = 0; i < net.leaves.size(); ++i) {
      std::vector<int> l = net.leaves[i].labels;
      std::sort(l.begin(), l.end());
      lab.push_back(l);
      alive.push_back(1);
      for (int x : l) holders[x].push_back((int)i);
    }
    n_live = (int)net.leaves.size();
  }

  bool summed(int l, int a, int b) const {
    for (int h : holders[l])
      if (h != a && h != b) return false;
    return true;
  }

  std::vector<int> result_labels(int a, int b) const {
    std::vector<int> u;
    std::set_union(lab[a].begin(), lab[a].end(), lab[b].begin(), lab[b].end(),
                   std::back_inserter(u));
    std::vector<int> out;
    for (int l : u)
      if (!summed(l, a, b)) out.push_back(l);
    return out;
  }

  int union_size(int a, int b) const {
    std::vector<int> u;
    std::set_union(lab[a].begin(), lab[a].end(), lab[b].begin(), lab[b].end(),
                   std::back_inserter(u));
    return (int)u.size();
  }

  int contract(int a, int b) {
    std::vector<int> r = result_labels(a, b);
    int id = (int)lab.size();
    for (int t : {a, b}) {
      for (int l : lab[t]) {
        auto& h = holders[l];
        h.erase(std::remove(h.begin(), h.end(), t), h.end());
      }
      alive[t] = 0;
    }
    for (int l : r) holders[l].push_back(id);
    lab.push_back(r);
    alive.push_back(1);
    steps.push_back({a, b});
    n_live -= 1;
    return id;
  }

  // Closes disconnected pieces (and final scalars) by outer products,
  // smallest tensors first.
  void finish() {
    while (n_live > 1) {
      int a = -1, b = -1;
      for (int t = 0; t < (int)lab.size(); ++t) {
        if (!alive[t]) continue;
        if (a < 0 || lab[t].size() < lab[a].size()) {
          b = a;
          a = t;
        } else if (b < 0 || lab[t].size() < lab[b].size()) {
          b = t;
        }
      }
      contract(a, b);
    }
  }
};

struct Cost {
  double flops = 0;     // sum 2^|A u B|
  double elems = 0;     // sum |A| + |B| + |C|
  int max_rank = 0;
  double score() const { return flops + elems; }
};

Cost cost_of(const Network& net, const std::vector<Step>& steps) {
  TNState st(net);
  Cost c;
  for (const Step& s : steps) {
    int u = st.union_size(s.a, s.b);
    double ea = std::ldexp(1.0, (int)st.lab[s.a].size());
    double eb = std::ldexp(1.0, (int)st.lab[s.b].size());
    int id = st.contract(s.a, s.b);
    int rc = (int)st.lab[id].size();
    c.flops += std::ldexp(1.0, u);
    c.elems += ea + eb + std::ldexp(1.0, rc);
    c.max_rank = std::max(c.max_rank, rc);
  }
  return c;
}

// Algorithm 2.  Threshold starts at -1; a randomly chosen wire is contracted
// when rank(C) - max(rank A, rank B) <= Threshold, which then resets to -1
// with the rejection count; after more than MaxRejections consecutive
// rejections the threshold grows by one.  A wire shared by more than two
// tensors (a hyperedge) contributes a random pair of its holders.
std::vector<Step> stoch_order(const Network& net, const qtc_plan_opts& o) {
  TNState st(net);
  SplitMix64 rng(o.seed);
  const int max_rej = o.max_rejections > 0 ? o.max_rejections : 10;
  int threshold = -1, rejections = 0;
  std::vector<int> active;
  while (st.n_live > 1) {
    active.clear();
    for (int l = 0; l < net.n_labels; ++l)
      if (st.holders[l].size() >= 2) active.push_back(l);
    if (active.empty()) {
      st.finish();
      break;
    }
    int w = active[rng.below(active.size())];
    const auto& hs = st.holders[w];
    int a, b;
    if (hs.size() == 2) {
      a = hs[0];
      b = hs[1];
    } else {
      size_t i = rng.below(hs.size());
      size_t j = rng.below(hs.size() - 1);
      if (j >= i) ++j;
      a = hs[i];
      b = hs[j];
    }
    int rc = (int)st.result_labels(a, b).size();
    int cost = rc - (int)std::max(st.lab[a].size(), st.lab[b].size());
    if (cost <= threshold) {
      st.contract(a, b);
      rejections = 0;
      threshold = -1;
    } else if (++rejections > max_rej) {
      threshold += 1;
      rejections = 0;
    }
  }
  return st.steps;
}

// Line graph of the network (one vertex per index, adjacent when a tensor
// holds both) as bitsets.
struct BitGraph {
  int n, words;
  std::vector<uint64_t> bits;
  explicit BitGraph(int n_) : n(n_), words((n_ + 63) / 64), bits((size_t)n_ * words, 0) {}
  uint64_t* row(int v) { return &bits[(size_t)v * words]; }
  const uint64_t* row(int v) const { return &bits[(size_t)v * words]; }
  void add(int a, int b) {
    row(a)[b >> 6] |= 1ull << (b & 63);
    row(b)[a >> 6] |= 1ull << (a & 63);
  }
  bool has(int a, int b) const { return (row(a)[b >> 6] >> (b & 63)) & 1; }
};

BitGraph line_graph(const Network& net) {
  BitGraph g(net.n_labels);
  for (const Leaf& leaf : net.leaves)
    for (size_t i = 0; i < leaf.labels.size(); ++i)
      for (size_t j = i + 1; j < leaf.labels.size(); ++j) g.add(leaf.labels[i], leaf.labels[j]);
  return g;
}

// Greedy min-fill elimination ordering with random tie-breaks (stands in for
// QuickBB's tree decomposition).  Returns the order and its width.
std::vector<int> min_fill_order(BitGraph g, SplitMix64& rng, int* width) {
  const int n = g.n, W = g.words;
  std::vector<char> alive(n, 1);
  std::vector<uint64_t> key(n);
  for (int v = 0; v < n; ++v) key[v] = rng.next();
  std::vector<long> fill(n, 0);
  std::vector<int> degree(n, 0);
  std::vector<char> dirty(n, 1);
  std::vector<int> order;
  order.reserve(n);
  std::vector<int> nb;
  *width = 0;
  auto neighbours = [&](int v, std::vector<int>& out) {
    out.clear();
    const uint64_t* r = g.row(v);
    for (int w = 0; w < W; ++w) {
      uint64_t x = r[w];
      while (x) {
        int b = __builtin_ctzll(x);
        out.push_back(w * 64 + b);
        x &= x - 1;
      }
    }
  };
  for (int it = 0; it < n; ++it) {
    for (int v = 0; v < n; ++v) {
      if (!alive[v] || !dirty[v]) continue;
      neighbours(v, nb);
      long f = 0;
      const uint64_t* rv = g.row(v);
      for (int u : nb) {
        const uint64_t* ru = g.row(u);
        long missing = 0;
        for (int w = 0; w < W; ++w) missing += __builtin_popcountll(rv[w] & ~ru[w]);
        f += missing - 1;  // u itself is in N(v) but not in N(u)
      }
      fill[v] = f / 2;
      degree[v] = (int)nb.size();
      dirty[v] = 0;
    }
    int best = -1;
    for (int v = 0; v < n; ++v) {
      if (!alive[v]) continue;
      if (best < 0 || fill[v] < fill[best] ||
          (fill[v] == fill[best] &&
           (degree[v] < degree[best] || (degree[v] == degree[best] && key[v] < key[best]))))
        best = v;
    }
    neighbours(best, nb);
    *width = std::max(*width, (int)nb.size());
    // connect the neighbours into a clique and drop `best`
    for (size_t i = 0; i < nb.size(); ++i)
      for (size_t j = i + 1; j < nb.size(); ++j) g.add(nb[i], nb[j]);
    for (int u : nb) {
      g.row(u)[best >> 6] &= ~(1ull << (best & 63));
      dirty[u] = 1;
      // neighbours of neighbours see new fill counts too
      const uint64_t* ru = g.row(u);
      for (int w = 0; w < W; ++w) {
        uint64_t x = ru[w];
        while (x) {
          dirty[w * 64 + __builtin_ctzll(x)] = 1;
          x &= x - 1;
        }
      }
    }
    std::fill(g.row(best), g.row(best) + W, 0ull);
    alive[best] = 0;
    order.push_back(best);
  }
  return order;
}

// Algorithm 1, step 3: eliminate the wires in order pi.  All tensors holding
// the wire are contracted pairwise (the pair with the smallest result first)
// until one remains; the wire is summed by the last pair.
std::vector<Step> eliminate(const Network& net, const std::vector<int>& order) {
  TNState st(net);
  for (int w : order) {
    while (st.holders[w].size() >= 2) {
      const auto& hs = st.holders[w];
      int ba = -1, bb = -1;
      long best_r = std::numeric_limits<long>::max(), best_s = 0;
      for (size_t i = 0; i < hs.size(); ++i)
        for (size_t j = i + 1; j < hs.size(); ++j) {
          long r = (long)st.result_labels(hs[i], hs[j]).size();
          long s = (long)(st.lab[hs[i]].size() + st.lab[hs[j]].size());
          if (r < best_r || (r == best_r && s < best_s)) {
            best_r = r;
            best_s = s;
            ba = hs[i];
            bb = hs[j];
          }
        }
      st.contract(ba, bb);
    }
  }
  st.finish();
  return st.steps;
}

// Per-step label layout.  A label's death is the step that sums it; every
// intermediate stores its labels by decreasing death step (the label that
// survives longest is bit 0), so operands of later steps share low bits.
void layout_labels(Plan& plan) {
  const Network& net = plan.net;
  const int L = (int)net.leaves.size();
  const int S = (int)plan.steps.size();
  TNState st(net);
  std::vector<int> death(net.n_labels, S);
  std::vector<std::vector<int>> result_sets;
  for (int s = 0; s < S; ++s) {
    const Step& stp = plan.steps[s];
    std::vector<int> u;
    std::set_union(st.lab[stp.a].begin(), st.lab[stp.a].end(), st.lab[stp.b].begin(),
                   st.lab[stp.b].end(), std::back_inserter(u));
    int id = st.contract(stp.a, stp.b);
    for (int l : u)
      if (!std::binary_search(st.lab[id].begin(), st.lab[id].end(), l)) death[l] = s;
    result_sets.push_back(st.lab[id]);
  }
  plan.labels.assign(L + S, {});
  for (int i = 0; i < L; ++i) plan.labels[i] = net.leaves[i].labels;
  for (int s = 0; s < S; ++s) {
    std::vector<int> r = result_sets[s];
    std::sort(r.begin(), r.end(), [&](int x, int y) {
      if (death[x] != death[y]) return death[x] > death[y];
      return x < y;
    });
    plan.labels[L + s] = r;
  }
  Cost c = cost_of(net, plan.steps);
  plan.max_rank = c.max_rank;
  plan.cmacs = c.flops;
  plan.bytes_c64 = 8.0 * c.elems;
}

}  // namespace

Plan make_plan(const Network& net, const qtc_plan_opts& o) {
  if (net.leaves.empty()) fail(QTC_ERR_INVALID, "empty network");
  Plan plan;
  plan.net = net;
  if (o.kind == QTC_ORDER_STOCH) {
    plan.steps = stoch_order(net, o);
  } else if (o.kind == QTC_ORDER_LG) {
    const int restarts = o.restarts > 0 ? o.restarts : 8;
    SplitMix64 rng(o.seed);
    BitGraph lgraph = line_graph(net);
    auto t0 = std::chrono::steady_clock::now();
    bool have = false;
    Cost best_cost;
    for (int r = 0; r < restarts; ++r) {
      int width = 0;
      std::vector<int> order = min_fill_order(lgraph, rng, &width);
      std::vector<Step> steps = eliminate(net, order);
      Cost c = cost_of(net, steps);
      if (!have || c.score() < best_cost.score() ||
          (c.score() == best_cost.score() && c.max_rank < best_cost.max_rank)) {
        have = true;
        best_cost = c;
        plan.steps = steps;
        plan.lg_width = width;
      }
      double ms = std::chrono::duration<double, std::milli>(
                      std::chrono::steady_clock::now() - t0).count();
      if (o.budget_ms > 0 && ms > o.budget_ms) break;
    }
  } else {
    fail(QTC_ERR_INVALID, "unknown ordering kind %d", o.kind);
  }
  if (plan.steps.empty()) {
    if (net.leaves.size() != 1) fail(QTC_ERR_INVALID, "internal: no steps for a multi-leaf network");
    fail(QTC_ERR_UNSUPPORTED, "a single-leaf network needs no contraction");
  }

  layout_labels(plan);
  return plan;
}

}  // namespace qtc
