// Lowering of a plan to the shared-memory op program: forward contractions
// (Eq. 1 with bit maps), the network scalar, and the adjoint sweep.
#include <algorithm>
#include <cstring>
#include <string>

#include "qtc_internal.h"

namespace qtc {

int GateTable::add(const GateSpec& s) {
  for (size_t i = 0; i < specs.size(); ++i) {
    const GateSpec& t = specs[i];
    if (t.kind == s.kind && t.conj == s.conj && t.slot == s.slot && t.coeff == s.coeff &&
        t.constant == s.constant)
      return (int)i;
  }
  specs.push_back(s);
  return (int)specs.size() - 1;
}

namespace {

int pos_in(const std::vector<int>& v, int x) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] == x) return (int)i;
  return -1;
}

// Fills the bit maps of out = sum over labels not in `lo` of in1 * in2.
bool encode_contract(SOp& op, const std::vector<int>& lo, const std::vector<int>& l1,
                     const std::vector<int>& l2) {
  if ((int)lo.size() > kMaxSmemRank || (int)l1.size() > kMaxSmemRank ||
      (int)l2.size() > kMaxSmemRank)
    return false;
  std::memset(op.p1, kAbsent, sizeof op.p1);
  std::memset(op.p2, kAbsent, sizeof op.p2);
  std::memset(op.y1, kAbsent, sizeof op.y1);
  std::memset(op.y2, kAbsent, sizeof op.y2);
  op.rc = (uint8_t)lo.size();
  for (size_t i = 0; i < lo.size(); ++i) {
    int a = pos_in(l1, lo[i]), b = pos_in(l2, lo[i]);
    op.p1[i] = a < 0 ? kAbsent : (uint8_t)a;
    op.p2[i] = b < 0 ? kAbsent : (uint8_t)b;
  }
  std::vector<int> summed;
  for (int x : l1)
    if (pos_in(lo, x) < 0) summed.push_back(x);
  for (int x : l2)
    if (pos_in(lo, x) < 0 && pos_in(l1, x) < 0) summed.push_back(x);
  if ((int)summed.size() > kMaxSmemRank) return false;
  op.ry = (uint8_t)summed.size();
  for (size_t j = 0; j < summed.size(); ++j) {
    int a = pos_in(l1, summed[j]), b = pos_in(l2, summed[j]);
    op.y1[j] = a < 0 ? kAbsent : (uint8_t)a;
    op.y2[j] = b < 0 ? kAbsent : (uint8_t)b;
  }
  return true;
}

struct Ref {
  int buf = -1;        // arena buffer id; else an absolute offset (table or global)
  uint32_t abs = 0;
  bool global = false; // abs is an element offset into the global work buffer
};

struct Pending {
  SOp op;
  Ref out, in1, in2;
};

// Places the arena buffers referenced by `ops` (first-fit decreasing over op
// index live ranges; a buffer written by op i and one read last by op i never
// share memory) and writes the resolved ops.  Buffers of at most
// `private_below` elements get memory of their own (no reuse at all with
// UINT32_MAX).  Returns the arena size.
uint32_t place_arena(const std::vector<Pending>& ops, const std::vector<uint32_t>& buf_size,
                     uint32_t table_elems, std::vector<SOp>& out, uint32_t private_below = 0) {
  const int B = (int)buf_size.size();
  std::vector<int> first(B, -1), last(B, -1);
  for (int i = 0; i < (int)ops.size(); ++i) {
    for (const Ref* r : {&ops[i].out, &ops[i].in1, &ops[i].in2}) {
      if (r->buf < 0) continue;
      if (first[r->buf] < 0) first[r->buf] = i;
      last[r->buf] = i;
    }
  }
  std::vector<int> order;
  for (int b = 0; b < B; ++b)
    if (first[b] >= 0) order.push_back(b);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (buf_size[a] != buf_size[b]) return buf_size[a] > buf_size[b];
    return a < b;
  });
  std::vector<uint32_t> offset(B, 0);
  std::vector<int> placed;
  uint32_t arena = 0;
  auto rounded = [&](int b) { return (buf_size[b] + 1u) & ~1u; };
  for (int b : order) {
    const uint32_t size = rounded(b);
    std::vector<std::pair<uint32_t, uint32_t>> busy;
    for (int q : placed)
      if (buf_size[b] <= private_below || buf_size[q] <= private_below ||
          !(last[q] < first[b] || last[b] < first[q]))
        busy.push_back({offset[q], offset[q] + rounded(q)});
    std::sort(busy.begin(), busy.end());
    uint32_t at = 0;
    for (auto& iv : busy) {
      if (at + size <= iv.first) break;
      at = std::max(at, iv.second);
    }
    offset[b] = at;
    placed.push_back(b);
    arena = std::max(arena, at + size);
  }
  auto resolve = [&](const Ref& r) { return r.buf < 0 ? r.abs : table_elems + offset[r.buf]; };
  for (const auto& p : ops) {
    SOp op = p.op;
    op.out = resolve(p.out);
    op.in1 = resolve(p.in1);
    op.in2 = resolve(p.in2);
    op.flags = (p.out.global ? SOPF_OUT_GLOBAL : 0) | (p.in1.global ? SOPF_IN1_GLOBAL : 0) |
               (p.in2.global ? SOPF_IN2_GLOBAL : 0);
    out.push_back(op);
  }
  return arena;
}

std::vector<char> needs_grad(const Plan& plan) {
  const int L = (int)plan.net.leaves.size();
  const int S = (int)plan.steps.size();
  std::vector<char> need(L + S, 0);
  for (int i = 0; i < L; ++i) need[i] = plan.net.leaves[i].spec.slot >= 0;
  for (int s = 0; s < S; ++s) need[L + s] = need[plan.steps[s].a] || need[plan.steps[s].b];
  return need;
}

}  // namespace

LoweredNet lower_smem(const Plan& plan, const std::vector<int>& leaf_gate,
                      const std::vector<uint32_t>& gate_val_off,
                      const std::vector<uint32_t>& gate_der_off, uint32_t table_elems,
                      bool want_grad, uint32_t max_elems, uint32_t private_below) {
  LoweredNet out;
  const int L = (int)plan.net.leaves.size();
  const int S = (int)plan.steps.size();
  const int T = L + S;
  const int root = T - 1;
  for (int t = 0; t < T; ++t)
    if ((int)plan.labels[t].size() > kMaxSmemRank) return out;
  const std::vector<char> need_grad = needs_grad(plan);

  // buffers: value of every intermediate, adjoint of every tensor that needs one
  std::vector<int> val_buf(T, -1), grad_buf(T, -1);
  std::vector<uint32_t> buf_size;
  for (int t = L; t < T; ++t) {
    val_buf[t] = (int)buf_size.size();
    buf_size.push_back(1u << plan.labels[t].size());
  }
  if (want_grad)
    for (int t = 0; t < T; ++t)
      if (need_grad[t]) {
        grad_buf[t] = (int)buf_size.size();
        buf_size.push_back(1u << plan.labels[t].size());
      }
  auto value_ref = [&](int t) {
    Ref r;
    if (t < L)
      r.abs = gate_val_off[leaf_gate[t]];
    else
      r.buf = val_buf[t];
    return r;
  };
  auto grad_ref = [&](int t) {
    Ref r;
    r.buf = grad_buf[t];
    return r;
  };

  std::vector<Pending> ops;
  for (int s = 0; s < S; ++s) {
    Pending p{};
    p.op.code = SOP_CONTRACT;
    const Step& st = plan.steps[s];
    if (!encode_contract(p.op, plan.labels[L + s], plan.labels[st.a], plan.labels[st.b]))
      return out;
    p.out = value_ref(L + s);
    p.in1 = value_ref(st.a);
    p.in2 = value_ref(st.b);
    ops.push_back(p);
  }
  {
    Pending p{};
    p.op.code = SOP_RESULT;
    p.in1 = value_ref(root);
    ops.push_back(p);
  }
  if (want_grad && need_grad[root]) {
    Pending seed{};
    seed.op.code = SOP_SEED;
    seed.out = grad_ref(root);
    ops.push_back(seed);
    for (int s = S - 1; s >= 0; --s) {
      const int c = L + s;
      const Step& st = plan.steps[s];
      const int pairs[2][2] = {{st.a, st.b}, {st.b, st.a}};
      for (const auto& pr : pairs) {
        int x = pr[0], y = pr[1];
        if (!need_grad[x]) continue;
        // adjoint of an operand: dS/dX = sum over the labels of C and Y not
        // in X of dS/dC * Y (holomorphic, no conjugation)
        Pending p{};
        p.op.code = SOP_CONTRACT;
        if (!encode_contract(p.op, plan.labels[x], plan.labels[c], plan.labels[y])) return out;
        p.out = grad_ref(x);
        p.in1 = grad_ref(c);
        p.in2 = value_ref(y);
        ops.push_back(p);
        if (x < L) {
          Pending g{};
          g.op.code = SOP_LEAFGRAD;
          g.op.rc = (uint8_t)plan.labels[x].size();
          g.in1 = grad_ref(x);
          g.in2.abs = gate_der_off[leaf_gate[x]];
          g.out.abs = (uint32_t)plan.net.leaves[x].spec.slot;
          ops.push_back(g);
        }
      }
    }
  }
  out.arena_elems = place_arena(ops, buf_size, table_elems, out.ops, private_below);
  out.fits = table_elems + out.arena_elems <= max_elems;
  return out;
}

// ---- graph lowering -----------------------------------------------------------

namespace {

// Bit maps of a global step as runs: bit i of `idx` goes to position pos[i]
// of the operand (-1: the operand does not carry it).
bool make_runs(const std::vector<int>& pos, GRuns& r) {
  std::memset(&r, 0, sizeof r);
  int i = 0;
  const int n = (int)pos.size();
  while (i < n) {
    if (pos[i] < 0) {
      ++i;
      continue;
    }
    int j = i + 1;
    while (j < n && pos[j] == pos[j - 1] + 1) ++j;
    if (r.n == kMaxRuns) return false;
    r.src[r.n] = (uint8_t)i;
    r.len[r.n] = (uint8_t)(j - i);
    r.dst[r.n] = (uint8_t)pos[i];
    r.n++;
    i = j;
  }
  return true;
}

uint32_t log2_floor(uint64_t x) {
  uint32_t r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

}  // namespace

// Fills the bit maps and chunking of C = sum over (A u B) - C of A * B.
// force_split: always reduce over chunks of the summed index (leaf adjoints).
// A chunk task covers about 2^task_terms_log2 multiply-adds.
bool encode_gstep(GStep& g, const std::vector<int>& lc, const std::vector<int>& la,
                  const std::vector<int>& lb, bool force_split, int task_terms_log2,
                  bool a_global, bool b_global, std::string* why) {
  std::vector<int> pa, pb, ya, yb;
  for (int x : lc) {
    pa.push_back(pos_in(la, x));
    pb.push_back(pos_in(lb, x));
  }
  std::vector<int> summed;
  for (int x : la)
    if (pos_in(lc, x) < 0) summed.push_back(x);
  for (int x : lb)
    if (pos_in(lc, x) < 0 && pos_in(la, x) < 0) summed.push_back(x);
  for (int x : summed) {
    ya.push_back(pos_in(la, x));
    yb.push_back(pos_in(lb, x));
  }
  if (lc.size() > 31 || summed.size() > 31) {
    *why = "a step's output or summed index exceeds 31 bits";
    return false;
  }
  g.rc = (uint8_t)lc.size();
  g.ry = (uint8_t)summed.size();
  if (!make_runs(pa, g.ca) || !make_runs(pb, g.cb) || !make_runs(ya, g.ya) ||
      !make_runs(yb, g.yb)) {
    *why = "a step's bit maps need more than 12 runs";
    return false;
  }
  const uint64_t nout = 1ull << g.rc, ny = 1ull << g.ry;
  if (nout <= kGRow && (force_split || nout * ny >= (1ull << 14))) {
    // small output, long sums: split the summed index over chunks
    uint64_t per = std::max<uint64_t>(256, (1ull << task_terms_log2) / nout);
    per = std::min<uint64_t>(per, kYTab);
    per = std::min<uint64_t>(per, ny);
    g.flags |= GSF_SPLIT;
    g.chunk = (uint32_t)per;
    g.n_chunks = (uint32_t)((ny + per - 1) / per);
  } else {
    const uint64_t rowlen = std::min<uint64_t>(nout, kGRow);
    const uint64_t rows = nout / rowlen;
    uint64_t per = 1;
    if (ny <= kYTab) {
      per = std::max<uint64_t>(1, (1ull << task_terms_log2) / (rowlen * ny));
      per = std::min<uint64_t>(per, kMaxChunkRows);
      per = std::min<uint64_t>(per, rows);
    }
    g.chunk = (uint32_t)per;
    g.n_chunks = (uint32_t)((rows + per - 1) / per);
  }
  // access forms: the summed index's lowest bits against the operands' own
  auto low_run = [](const GRuns& r) {
    return (r.n > 0 && r.src[0] == 0 && r.dst[0] == 0) ? (int)r.len[0] : 0;
  };
  const int la0 = low_run(g.ya), lb0 = low_run(g.yb);
  if (a_global && b_global && g.ry >= 1 && la0 >= 1 && lb0 >= 1 && !(g.flags & GSF_SPLIT))
    g.flags |= GSF_YPAIR;
  if (a_global && b_global && (g.flags & GSF_SPLIT) && std::max(la0, lb0) >= 3)
    g.flags |= GSF_LANES_Y;
  // short sums over rows: groups of rows along output labels one operand
  // lacks, that operand read once per group (the other's loads all in flight)
  if (!(g.flags & (GSF_SPLIT | GSF_YPAIR)) && ny <= 4) {
    const int G = grs_fix_bits((uint32_t)ny);
    const int row0 = log2_floor(kGRow), nrow_bits = g.rc - row0;
    if (nout >= ((uint64_t)kGRow << G)) {
      std::vector<int> zs, xs;   // row bits (relative) missing from A, from B
      for (int i = 0; i < nrow_bits; ++i) {
        if (pa[row0 + i] < 0) zs.push_back(i);
        if (pb[row0 + i] < 0) xs.push_back(i);
      }
      const bool fix_b = (int)xs.size() >= G && xs.size() >= zs.size();
      const bool fix_a = !fix_b && (int)zs.size() >= G;
      if (fix_a || fix_b) {
        const std::vector<int>& sel = fix_b ? xs : zs;
        std::vector<int> order(sel.begin(), sel.begin() + G);
        for (int i = 0; i < nrow_bits; ++i)
          if (std::find(order.begin(), order.end(), i) == order.end()) order.push_back(i);
        GRuns rows;
        if (make_runs(order, rows)) {
          const uint64_t nrows = nout / kGRow, grp = 1ull << G;
          const uint64_t per = std::min<uint64_t>(std::max<uint64_t>(g.chunk, grp), nrows);
          g.rows = rows;
          g.share = fix_b ? GRS_FIXB : GRS_FIXA;
          g.chunk = (uint32_t)per;
          g.n_chunks = (uint32_t)(nrows / per);
          g.flags |= GSF_ROWS;
        }
      }
    }
  }
  // long sums over rows: take rows four at a time along output labels missing
  // from one operand, so the four rows read fewer distinct elements per term
  // (with paired loads too)
  if (a_global && b_global && !(g.flags & GSF_SPLIT) && ny >= 8 && ny <= kYTab &&
      nout >= 4 * kGRow) {
    const int row0 = log2_floor(kGRow), nrow_bits = g.rc - row0;
    std::vector<int> zs, xs;   // row bits (relative) missing from A, from B
    for (int i = 0; i < nrow_bits; ++i) {
      if (pa[row0 + i] < 0) zs.push_back(i);
      else if (pb[row0 + i] < 0) xs.push_back(i);
    }
    int b0 = -1, b1 = -1;
    uint8_t share = 0;
    if (!zs.empty() && !xs.empty()) {
      b0 = zs[0], b1 = xs[0], share = GRS_ZX;
    } else if (zs.size() >= 2) {
      b0 = zs[0], b1 = zs[1], share = GRS_ZZ;
    } else if (xs.size() >= 2) {
      b0 = xs[0], b1 = xs[1], share = GRS_XX;
    }
    if (share) {
      std::vector<int> order = {b0, b1};
      for (int i = 0; i < nrow_bits; ++i)
        if (i != b0 && i != b1) order.push_back(i);
      GRuns rows;
      if (make_runs(order, rows)) {
        const uint64_t nrows = nout / kGRow;
        const uint64_t per = std::min<uint64_t>(std::max<uint64_t>(g.chunk, 4), nrows);
        g.rows = rows;
        g.share = share;
        g.chunk = (uint32_t)per;
        g.n_chunks = (uint32_t)(nrows / per);
        g.flags |= GSF_ROWS;
      }
    }
  }
  return true;
}

// A step as a batched complex GEMM for the tensor cores: C labels are batch
// (in both operands) or free in exactly one operand, summed labels are in
// both operands.  Eligible when M and N have >= 64 entries and K >= 8.
bool encode_tstep(TStep& t, const std::vector<int>& lc, const std::vector<int>& la,
                  const std::vector<int>& lb) {
  std::vector<int> bl, ml, nl, kl;
  for (int x : lc) {
    const bool in_a = pos_in(la, x) >= 0, in_b = pos_in(lb, x) >= 0;
    if (in_a && in_b) bl.push_back(x);
    else if (in_a) ml.push_back(x);
    else if (in_b) nl.push_back(x);
    else return false;  // an output label in neither operand
  }
  for (int x : la)
    if (pos_in(lc, x) < 0) {
      if (pos_in(lb, x) < 0) return false;  // summed in one operand only
      kl.push_back(x);
    }
  for (int x : lb)
    if (pos_in(lc, x) < 0 && pos_in(la, x) < 0) return false;
  if (ml.size() < 6 || nl.size() < 6 || kl.size() < 3) return false;
  if (ml.size() > 24 || nl.size() > 24 || kl.size() > 24 || bl.size() > 24) return false;
  std::memset(&t, 0, sizeof t);
  auto pos = [](const std::vector<int>& labels, const std::vector<int>& in) {
    std::vector<int> p;
    for (int x : labels) p.push_back(pos_in(in, x));
    return p;
  };
  bool ok = make_runs(pos(ml, la), t.am) && make_runs(pos(kl, la), t.ak) &&
            make_runs(pos(bl, la), t.ab) && make_runs(pos(kl, lb), t.bk) &&
            make_runs(pos(nl, lb), t.bn) && make_runs(pos(bl, lb), t.bbt) &&
            make_runs(pos(ml, lc), t.cm) && make_runs(pos(nl, lc), t.cn) &&
            make_runs(pos(bl, lc), t.cb);
  if (!ok) return false;
  t.mb = (uint8_t)ml.size();
  t.kb = (uint8_t)kl.size();
  t.nb = (uint8_t)nl.size();
  t.bb = (uint8_t)bl.size();
  t.m_tiles = (uint32_t)(((1ull << t.mb) + kTcRows - 1) / kTcRows);
  t.n_tiles = (uint32_t)((1ull << t.nb) / kTcCols);
  return true;
}

// ---- global work-buffer placement by live range ------------------------------

namespace {

struct GRef {
  uint32_t* off;   // element offset in the work buffer (a buffer's start)
  bool write;
};

// Every work-buffer reference of a unit, with whether the unit writes it.
std::vector<GRef> unit_refs(GUnit& u) {
  std::vector<GRef> r;
  if (u.kind == GT_SMEM) {
    for (SOp& op : u.ops) {
      if (op.flags & SOPF_OUT_GLOBAL) r.push_back({&op.out, true});
      if (op.flags & SOPF_IN1_GLOBAL) r.push_back({&op.in1, false});
      if (op.flags & SOPF_IN2_GLOBAL) r.push_back({&op.in2, false});
    }
  } else if (u.kind == GT_CHUNK) {
    GStep& st = u.step;
    if (!(st.flags & GSF_A_TABLE)) r.push_back({&st.a_off, false});
    if (!(st.flags & GSF_B_TABLE)) r.push_back({&st.b_off, false});
    if (!(st.flags & GSF_LEAFGRAD)) r.push_back({&st.c_off, true});
    if (st.flags & GSF_SPLIT) r.push_back({&st.partial_off, true});
  } else {
    r.push_back({&u.tstep.a_off, false});
    r.push_back({&u.tstep.b_off, false});
    r.push_back({&u.tstep.c_off, true});
  }
  return r;
}

}  // namespace

void place_global_buffers(NetGraph& ng, const std::vector<uint64_t>& vbase,
                          const std::vector<uint64_t>& vsize, bool add_deps) {
  const int B = (int)vbase.size();
  const int U = (int)ng.units.size();
  if (B == 0) return;
  auto buffer_of = [&](uint32_t off) {
    const int b = (int)(std::upper_bound(vbase.begin(), vbase.end(), (uint64_t)off) -
                        vbase.begin()) - 1;
    if (b < 0 || off >= vbase[b] + vsize[b]) fail(QTC_ERR_INVALID, "internal: global offset %u", off);
    return b;
  };
  // live range of each buffer in unit (creation) order, its writers and all
  // units that touch it
  std::vector<int> first(B, -1), last(B, -1);
  std::vector<std::vector<int>> writers(B), users(B);
  for (int i = 0; i < U; ++i)
    for (const GRef& r : unit_refs(ng.units[i])) {
      const int b = buffer_of(*r.off);
      if (first[b] < 0) first[b] = i;
      last[b] = i;
      if (users[b].empty() || users[b].back() != i) users[b].push_back(i);
      if (r.write && (writers[b].empty() || writers[b].back() != i)) writers[b].push_back(i);
    }
  // ancestors of every unit (dependencies point to earlier units)
  const int W = (U + 63) / 64;
  std::vector<uint64_t> anc((size_t)U * W, 0);
  for (int i = 0; i < U; ++i)
    for (int d : ng.units[i].deps) {
      if (d < 0 || d >= i) continue;
      uint64_t* a = &anc[(size_t)i * W];
      const uint64_t* ad = &anc[(size_t)d * W];
      for (int k = 0; k < W; ++k) a[k] |= ad[k];
      a[d / 64] |= 1ull << (d % 64);
    }
  auto is_anc = [&](int a, int of) { return (anc[(size_t)of * W + a / 64] >> (a % 64)) & 1; };
  // q's memory may be taken by b without a new dependency when every unit
  // that touches q already precedes every writer of b
  auto ordered_before = [&](int q, int b) {
    if (!(last[q] < first[b])) return false;
    if (add_deps) return true;   // the dependencies are added below
    for (int w : writers[b])
      for (int u : users[q])
        if (u != w && !is_anc(u, w)) return false;
    return true;
  };
  // first fit, largest buffers first; two buffers share memory only when
  // one's every use is ordered before the other's writes
  std::vector<int> order;
  for (int b = 0; b < B; ++b)
    if (first[b] >= 0) order.push_back(b);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (vsize[a] != vsize[b]) return vsize[a] > vsize[b];
    return a < b;
  });
  std::vector<uint64_t> at(B, 0);
  std::vector<int> placed;
  uint64_t peak = 0;
  for (int b : order) {
    std::vector<std::pair<uint64_t, uint64_t>> busy;
    for (int q : placed)
      if (!ordered_before(q, b) && !ordered_before(b, q)) busy.push_back({at[q], at[q] + vsize[q]});
    std::sort(busy.begin(), busy.end());
    uint64_t pos = 0;
    for (auto& iv : busy) {
      if (pos + vsize[b] <= iv.first) break;
      pos = std::max(pos, iv.second);
    }
    at[b] = pos;
    placed.push_back(b);
    peak = std::max(peak, pos + vsize[b]);
  }
  if (add_deps) {
    // write after read: a buffer's writers start only after every unit that
    // touched an earlier buffer in the same memory has finished
    for (int b : placed)
      for (int q : placed) {
        if (q == b || !(last[q] < first[b])) continue;
        if (at[q] >= at[b] + vsize[b] || at[b] >= at[q] + vsize[q]) continue;
        for (int w : writers[b])
          for (int u : users[q])
            if (u != w) ng.units[w].deps.push_back(u);
      }
    // depths again (dependencies still point to earlier units)
    for (int i = 0; i < U; ++i) {
      GUnit& u = ng.units[i];
      std::sort(u.deps.begin(), u.deps.end());
      u.deps.erase(std::unique(u.deps.begin(), u.deps.end()), u.deps.end());
      int depth = 0;
      for (int d : u.deps) {
        if (d >= i) fail(QTC_ERR_INVALID, "internal: a dependency on a later unit");
        depth = std::max(depth, ng.units[d].depth + 1);
      }
      u.depth = depth;
    }
  }
  for (int i = 0; i < U; ++i)
    for (const GRef& r : unit_refs(ng.units[i])) {
      const int b = buffer_of(*r.off);
      *r.off = (uint32_t)(at[b] + (*r.off - vbase[b]));
    }
  ng.global_elems = peak;
  ng.buffers.clear();
  for (int b : placed) ng.buffers.push_back({at[b], vsize[b], first[b], last[b], writers[b], users[b]});
}

// Host check of a placement: every pair of buffers that share memory is
// ordered (all units touching the earlier one are ancestors of every writer
// of the later one) and no two live buffers overlap.
void check_global_placement(const NetGraph& ng) {
  const int U = (int)ng.units.size();
  const int W = (U + 63) / 64;
  std::vector<uint64_t> anc((size_t)U * W, 0);
  for (int i = 0; i < U; ++i)
    for (int d : ng.units[i].deps) {
      uint64_t* a = &anc[(size_t)i * W];
      const uint64_t* ad = &anc[(size_t)d * W];
      for (int k = 0; k < W; ++k) a[k] |= ad[k];
      a[d / 64] |= 1ull << (d % 64);
    }
  auto is_anc = [&](int a, int of) { return (anc[(size_t)of * W + a / 64] >> (a % 64)) & 1; };
  const auto& bs = ng.buffers;
  for (size_t x = 0; x < bs.size(); ++x)
    for (size_t y = 0; y < bs.size(); ++y) {
      if (x == y) continue;
      const auto& p = bs[x];
      const auto& q = bs[y];
      if (p.at >= q.at + q.size || q.at >= p.at + p.size) continue;
      if (!(p.last < q.first))
        if (!(q.last < p.first))
          fail(QTC_ERR_INVALID, "internal: live global buffers share memory");
      if (p.last < q.first)
        for (int w : q.writers)
          for (int u : p.users)
            if (u != w && !is_anc(u, w))
              fail(QTC_ERR_INVALID, "internal: a write to reused memory is not ordered after "
                                    "the earlier reads");
    }
}

NetGraph lower_graph(const Plan& plan, const std::vector<int>& leaf_gate,
                     const std::vector<uint32_t>& gate_val_off,
                     const std::vector<uint32_t>& gate_der_off, uint32_t table_elems,
                     bool want_grad, const GraphLimits& lim) {
  NetGraph ng;
  const int L = (int)plan.net.leaves.size();
  const int S = (int)plan.steps.size();
  const int T = L + S;
  const int root = T - 1;
  const std::vector<char> need_grad = needs_grad(plan);
  auto rank = [&](int t) { return (int)plan.labels[t].size(); };
  auto size = [&](int t) { return (uint64_t)1 << rank(t); };
  std::vector<int> consumer(T, -1);
  for (int s = 0; s < S; ++s) consumer[plan.steps[s].a] = consumer[plan.steps[s].b] = s;
  std::vector<char> bigstep(S, 0);
  for (int s = 0; s < S; ++s) {
    const Step& st = plan.steps[s];
    bigstep[s] = rank(st.a) > lim.small_rank || rank(st.b) > lim.small_rank ||
                 rank(L + s) > lim.small_rank;
  }

  // subtrees of small steps (walked from the root down), capped in size
  std::vector<int> sub(S, -1), sub_root;
  std::vector<uint64_t> sub_size;
  for (int s = S - 1; s >= 0; --s) {
    if (bigstep[s]) continue;
    const int c = consumer[L + s];
    if (c >= 0 && !bigstep[c] && sub_size[sub[c]] + size(L + s) <= lim.subtree_elems) {
      sub[s] = sub[c];
      sub_size[sub[c]] += size(L + s);
    } else {
      sub[s] = (int)sub_root.size();
      sub_root.push_back(s);
      sub_size.push_back(size(L + s));
    }
  }
  const int K = (int)sub_root.size();
  std::vector<std::vector<int>> sub_steps(K);
  for (int s = 0; s < S; ++s)
    if (sub[s] >= 0) sub_steps[sub[s]].push_back(s);

  // tensors in global memory: outputs of large steps and of subtree roots
  // (except the network root when a subtree produces it)
  std::vector<char> in_global(T, 0);
  for (int s = 0; s < S; ++s)
    if (bigstep[s] || (sub_root[sub[s]] == s && L + s != root)) in_global[L + s] = 1;
  std::vector<int64_t> val_g(T, -1), grad_g(T, -1);
  // Every global tensor first gets a region of its own in a virtual layout
  // (vbase, vsize); place_global_buffers then overlaps regions whose live
  // ranges do not meet and rewrites the offsets.
  uint64_t gsize = 0;
  std::vector<uint64_t> vbase, vsize;
  auto galloc = [&](uint64_t elems) {
    const uint64_t at = gsize;
    vbase.push_back(at);
    vsize.push_back((elems + 63) & ~uint64_t(63));
    gsize += vsize.back();
    return (int64_t)at;
  };
  for (int t = L; t < T; ++t)
    if (in_global[t]) val_g[t] = galloc(size(t));
  if (want_grad)
    for (int t = L; t < T; ++t)
      if (in_global[t] && need_grad[t]) grad_g[t] = galloc(size(t));

  std::vector<int> producer_val(T, -1), producer_grad(T, -1);
  // recomputed segments start after the adjoint sweep reaches them (>= 0:
  // the unit every forward unit emitted now also waits for)
  int recompute_after = -1;
  auto add_unit = [&](GUnit&& u) {
    int depth = 0;
    std::sort(u.deps.begin(), u.deps.end());
    u.deps.erase(std::unique(u.deps.begin(), u.deps.end()), u.deps.end());
    for (int d : u.deps) depth = std::max(depth, ng.units[d].depth + 1);
    u.depth = depth;
    ng.units.push_back(std::move(u));
    return (int)ng.units.size() - 1;
  };
  auto fail_net = [&](const std::string& why) {
    ng.fits = false;
    ng.why = why;
    return ng;
  };

  // ---- forward ----
  // Shared-memory program of a subtree; `reverse` adds the adjoint sweep
  // (recomputing the subtree's values first).
  auto subtree_unit = [&](int k, bool reverse) -> bool {
    const std::vector<int>& steps = sub_steps[k];
    const int rs = sub_root[k];
    std::vector<int> val_buf(T, -1), grad_buf(T, -1);
    std::vector<uint32_t> buf_size;
    GUnit u;
    u.kind = GT_SMEM;
    if (!reverse && recompute_after >= 0) u.deps.push_back(recompute_after);
    auto value_ref = [&](int t) {
      Ref r;
      if (t < L) {
        r.abs = gate_val_off[leaf_gate[t]];
      } else if (in_global[t] && !(t == L + rs && !reverse)) {
        r.global = true;
        r.abs = (uint32_t)val_g[t];
        if (t != L + rs) u.deps.push_back(producer_val[t]);
      } else {
        if (val_buf[t] < 0) {
          val_buf[t] = (int)buf_size.size();
          buf_size.push_back((uint32_t)size(t));
        }
        r.buf = val_buf[t];
      }
      return r;
    };
    auto grad_ref = [&](int t) {
      Ref r;
      if (t >= L && in_global[t] && t != L + rs) {
        r.global = true;
        r.abs = (uint32_t)grad_g[t];
      } else if (t == L + rs && in_global[t]) {
        r.global = true;
        r.abs = (uint32_t)grad_g[t];
        u.deps.push_back(producer_grad[t]);
      } else {
        if (grad_buf[t] < 0) {
          grad_buf[t] = (int)buf_size.size();
          buf_size.push_back((uint32_t)size(t));
        }
        r.buf = grad_buf[t];
      }
      return r;
    };
    std::vector<Pending> ops;
    for (int s : steps) {
      if (reverse && s == rs) continue;  // the root's own value is not needed
      const Step& st = plan.steps[s];
      Pending p{};
      p.op.code = SOP_CONTRACT;
      if (!encode_contract(p.op, plan.labels[L + s], plan.labels[st.a], plan.labels[st.b]))
        return false;
      p.in1 = value_ref(st.a);
      p.in2 = value_ref(st.b);
      if (s == rs && in_global[L + s]) {
        p.out.global = true;
        p.out.abs = (uint32_t)val_g[L + s];
      } else {
        p.out = value_ref(L + s);
      }
      ops.push_back(p);
    }
    if (!reverse && L + rs == root) {
      Pending p{};
      p.op.code = SOP_RESULT;
      p.in1 = value_ref(root);
      ops.push_back(p);
    }
    if (reverse) {
      if (L + rs == root) {
        Pending seed{};
        seed.op.code = SOP_SEED;
        seed.out = grad_ref(root);
        ops.push_back(seed);
      }
      for (auto it = steps.rbegin(); it != steps.rend(); ++it) {
        const int s = *it;
        const int c = L + s;
        const Step& st = plan.steps[s];
        const int pairs[2][2] = {{st.a, st.b}, {st.b, st.a}};
        for (const auto& pr : pairs) {
          const int x = pr[0], y = pr[1];
          if (!need_grad[x]) continue;
          Pending p{};
          p.op.code = SOP_CONTRACT;
          if (!encode_contract(p.op, plan.labels[x], plan.labels[c], plan.labels[y]))
            return false;
          p.in1 = grad_ref(c);
          p.in2 = value_ref(y);
          p.out = grad_ref(x);
          ops.push_back(p);
          if (x < L) {
            Pending g{};
            g.op.code = SOP_LEAFGRAD;
            g.op.rc = (uint8_t)plan.labels[x].size();
            g.in1 = grad_ref(x);
            g.in2.abs = gate_der_off[leaf_gate[x]];
            g.out.abs = (uint32_t)plan.net.leaves[x].spec.slot;
            ops.push_back(g);
          } else if (in_global[x]) {
            producer_grad[x] = (int)ng.units.size();
          }
        }
      }
    }
    u.arena_elems = place_arena(ops, buf_size, table_elems, u.ops);
    if (u.arena_elems > lim.arena_elems) return false;
    const int id = add_unit(std::move(u));
    if (!reverse && in_global[L + rs]) producer_val[L + rs] = id;
    return true;
  };

  auto gstep_unit = [&](int lc_t, const std::vector<int>& lc, int a, const std::vector<int>& la,
                        Ref ra, int b, const std::vector<int>& lb, Ref rb, int64_t c_off,
                        std::vector<int> deps, int leaf_for_grad) -> int {
    GUnit u;
    if (lim.tensor_cores && leaf_for_grad < 0 && ra.global && rb.global &&
        encode_tstep(u.tstep, lc, la, lb)) {
      u.kind = GT_TC;
      u.tstep.c_off = (uint32_t)c_off;
      u.tstep.a_off = ra.abs;
      u.tstep.b_off = rb.abs;
      u.target = (uint32_t)(((uint64_t)u.tstep.m_tiles * u.tstep.n_tiles) << u.tstep.bb);
      u.deps = std::move(deps);
      return add_unit(std::move(u));
    }
    u.kind = GT_CHUNK;
    std::memset(&u.step, 0, sizeof u.step);
    std::string why;
    if (!encode_gstep(u.step, lc, la, lb, leaf_for_grad >= 0, lim.task_terms_log2, ra.global,
                      rb.global, &why)) {
      ng.fits = false;
      ng.why = why;
      return -1;
    }
    (void)lc_t;
    (void)a;
    (void)b;
    if (leaf_for_grad >= 0) u.step.flags |= GSF_LEAFGRAD;
    const bool two_global = ra.global && rb.global;
    const int tm = lim.tile_mode;
    if (tm == 2 || tm == 4 || (tm == 1 && (two_global || (u.step.flags & GSF_SPLIT))) ||
        (tm == 3 && u.step.ry >= 3)) {
      GStep tiled = u.step;
      tiled.flags &= (uint16_t)~(GSF_SPLIT | GSF_YPAIR | GSF_LANES_Y);
      if (encode_tile(tiled, lc, la, lb, !ra.global, !rb.global, lim.elem, lim.task_terms_log2,
                      tm >= 3))
        u.step = tiled;
    }
    u.step.c_off = (uint32_t)std::max<int64_t>(c_off, 0);
    if (ra.global) u.step.a_off = ra.abs;
    else { u.step.a_off = ra.abs; u.step.flags |= GSF_A_TABLE; }
    if (rb.global) u.step.b_off = rb.abs;
    else { u.step.b_off = rb.abs; u.step.flags |= GSF_B_TABLE; }
    if (leaf_for_grad >= 0) {
      if (!(u.step.flags & GSF_SPLIT)) {
        // the leaf gradient is always a reduction to <= 16 outputs
        ng.fits = false;
        ng.why = "internal: a leaf adjoint that is not a split reduction";
        return -1;
      }
      u.step.der_off = gate_der_off[leaf_gate[leaf_for_grad]];
      u.step.slot = plan.net.leaves[leaf_for_grad].spec.slot;
    }
    if (u.step.flags & GSF_SPLIT) {
      const uint32_t pbits = (u.step.flags & GSF_TILE) ? u.step.tile.nfc : u.step.rc;
      u.step.partial_off = (uint32_t)galloc((uint64_t)u.step.n_chunks << pbits);
      u.target = 1;
    } else {
      u.target = u.step.n_chunks;
    }
    u.deps = std::move(deps);
    return add_unit(std::move(u));
  };

  auto value_ref_global = [&](int t, std::vector<int>& deps) {
    Ref r;
    if (t < L) {
      r.abs = gate_val_off[leaf_gate[t]];
    } else {
      r.global = true;
      r.abs = (uint32_t)val_g[t];
      deps.push_back(producer_val[t]);
    }
    return r;
  };

  // forward units in step order: a subtree when its last step is reached
  std::vector<char> sub_done(K, 0);
  for (int s = 0; s < S; ++s) {
    if (bigstep[s]) {
      const Step& st = plan.steps[s];
      std::vector<int> deps;
      Ref ra = value_ref_global(st.a, deps);
      Ref rb = value_ref_global(st.b, deps);
      const int id = gstep_unit(L + s, plan.labels[L + s], st.a, plan.labels[st.a], ra, st.b,
                                plan.labels[st.b], rb, val_g[L + s], deps, -1);
      if (id < 0) return ng;
      producer_val[L + s] = id;
    } else if (sub_root[sub[s]] == s) {
      if (!subtree_unit(sub[s], false)) return fail_net("a subtree does not fit in shared memory");
    }
  }
  if (in_global[root]) {
    // the root comes from a large step: read it (and seed the adjoint)
    GUnit u;
    u.kind = GT_SMEM;
    Pending p{};
    p.op.code = SOP_RESULT;
    p.in1.global = true;
    p.in1.abs = (uint32_t)val_g[root];
    std::vector<Pending> ops{p};
    if (want_grad && need_grad[root]) {
      Pending seed{};
      seed.op.code = SOP_SEED;
      seed.out.global = true;
      seed.out.abs = (uint32_t)grad_g[root];
      ops.push_back(seed);
    }
    u.deps.push_back(producer_val[root]);
    place_arena(ops, {}, table_elems, u.ops);
    const int id = add_unit(std::move(u));
    producer_grad[root] = id;
  }

  // ---- checkpoint segments (gradient runs whose stored values exceed the cap)
  // The steps that write global tensors are cut, in step order, into
  // segments of about equal output size.  A global value used by a later
  // segment is a checkpoint and stays stored; one whose forward consumer is in
  // its own segment (the last segment excepted) is dropped after that use and
  // computed again when the adjoint sweep reaches its segment, so only the
  // checkpoints and one segment's values are held at a time.
  const int n_seg = want_grad ? std::max(1, lim.checkpoint_segments) : 1;
  ng.checkpoint_segments = n_seg;
  std::vector<int> seg(S, 0);
  std::vector<char> dropped(T, 0);
  if (n_seg > 1) {
    auto produces = [&](int s) { return bigstep[s] || (sub_root[sub[s]] == s && in_global[L + s]); };
    double total = 0;
    for (int s = 0; s < S; ++s)
      if (produces(s)) total += (double)size(L + s);
    double run = 0;
    int j = 0;
    for (int s = 0; s < S; ++s) {
      if (!bigstep[s] && sub_root[sub[s]] != s) continue;
      seg[s] = j;
      if (produces(s)) {
        run += (double)size(L + s);
        if (run >= (j + 1) * total / n_seg && j < n_seg - 1) ++j;
      }
    }
    auto seg_of = [&](int s) { return bigstep[s] ? seg[s] : seg[sub_root[sub[s]]]; };
    for (int s = 0; s < S; ++s) {
      const int t = L + s;
      if (!in_global[t] || t == root || !produces(s)) continue;
      const int c = consumer[t];
      if (seg[s] < n_seg - 1 && c >= 0 && seg_of(c) == seg[s]) dropped[t] = 1;
    }
  }
  // the segment's dropped values again, in step order, into fresh buffers
  auto recompute_segment = [&](int j) -> bool {
    // after the sweep so far: its memory can then be reused for the values
    recompute_after = ng.units.empty() ? -1 : (int)ng.units.size() - 1;
    for (int s = 0; s < S; ++s) {
      if (seg[s] != j || !dropped[L + s]) continue;
      if (bigstep[s]) {
        const Step& st = plan.steps[s];
        std::vector<int> deps;
        if (recompute_after >= 0) deps.push_back(recompute_after);
        Ref ra = value_ref_global(st.a, deps);
        Ref rb = value_ref_global(st.b, deps);
        val_g[L + s] = galloc(size(L + s));
        const int id = gstep_unit(L + s, plan.labels[L + s], st.a, plan.labels[st.a], ra, st.b,
                                  plan.labels[st.b], rb, val_g[L + s], deps, -1);
        if (id < 0) return false;
        producer_val[L + s] = id;
      } else if (sub_root[sub[s]] == s) {
        val_g[L + s] = galloc(size(L + s));
        if (!subtree_unit(sub[s], false)) {
          ng.fits = false;
          ng.why = "a subtree does not fit in shared memory";
          return false;
        }
      }
    }
    ng.recomputed_segments += 1;
    recompute_after = -1;
    return true;
  };

  // ---- adjoint sweep, in reverse step order ----
  if (want_grad && need_grad[root]) {
    int entered = n_seg - 1;
    for (int s = S - 1; s >= 0; --s) {
      if (n_seg > 1 && (bigstep[s] || sub_root[sub[s]] == s) && seg[s] < entered) {
        entered = seg[s];
        if (!recompute_segment(entered)) return ng;
      }
      if (bigstep[s]) {
        const int c = L + s;
        const Step& st = plan.steps[s];
        const int pairs[2][2] = {{st.a, st.b}, {st.b, st.a}};
        for (const auto& pr : pairs) {
          const int x = pr[0], y = pr[1];
          if (!need_grad[x]) continue;
          std::vector<int> deps{producer_grad[c]};
          Ref rg;
          rg.global = true;
          rg.abs = (uint32_t)grad_g[c];
          Ref ry = value_ref_global(y, deps);
          const int id = gstep_unit(x, plan.labels[x], c, plan.labels[c], rg, y, plan.labels[y],
                                    ry, x < L ? -1 : grad_g[x], deps, x < L ? x : -1);
          if (id < 0) return ng;
          if (x >= L) producer_grad[x] = id;
        }
      } else if (sub_root[sub[s]] == s && need_grad[L + s]) {
        if (!subtree_unit(sub[s], true)) return fail_net("a subtree does not fit in shared memory");
      }
    }
  }
  for (const GUnit& u : ng.units)
    for (int d : u.deps)
      if (d < 0) return fail_net("internal: a dependency without a producer");
  if (gsize >> 32) return fail_net("a network's global intermediates exceed 2^32 elements");
  ng.global_elems = gsize;
  ng.unshared_elems = gsize;
  if (lim.reuse_global) place_global_buffers(ng, vbase, vsize, lim.reuse_with_deps);
  (void)sub_done;
  return ng;
}

}  // namespace qtc
