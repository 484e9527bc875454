// Lowering of a plan to the shared-memory op program: forward contractions
// (Eq. 1 with bit maps), the network scalar, and the adjoint sweep.
#include <algorithm>
#include <cstring>

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
  int buf = -1;        // arena buffer id, or -1 for an absolute table offset
  uint32_t abs = 0;
};

struct Pending {
  SOp op;
  Ref out, in1, in2;
};

}  // namespace

LoweredNet lower_smem(const Plan& plan, const std::vector<int>& leaf_gate,
                      const std::vector<uint32_t>& gate_val_off,
                      const std::vector<uint32_t>& gate_der_off, uint32_t table_elems,
                      bool want_grad, uint32_t max_elems) {
  LoweredNet out;
  const int L = (int)plan.net.leaves.size();
  const int S = (int)plan.steps.size();
  const int T = L + S;
  const int root = T - 1;
  std::vector<char> need_grad(T, 0);
  for (int i = 0; i < L; ++i) need_grad[i] = plan.net.leaves[i].spec.slot >= 0;
  for (int s = 0; s < S; ++s)
    need_grad[L + s] = need_grad[plan.steps[s].a] || need_grad[plan.steps[s].b];

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

  // live intervals of the arena buffers over the op sequence
  const int B = (int)buf_size.size();
  std::vector<int> first(B, -1), last(B, -1);
  for (int i = 0; i < (int)ops.size(); ++i) {
    for (const Ref* r : {&ops[i].out, &ops[i].in1, &ops[i].in2}) {
      if (r->buf < 0) continue;
      if (first[r->buf] < 0) first[r->buf] = i;
      last[r->buf] = i;
    }
  }
  // first-fit decreasing placement (sizes rounded to 2 elements)
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
  for (int b : order) {
    uint32_t size = (buf_size[b] + 1u) & ~1u;
    std::vector<std::pair<uint32_t, uint32_t>> busy;
    for (int q : placed)
      if (!(last[q] < first[b] || last[b] < first[q]))
        busy.push_back({offset[q], offset[q] + ((buf_size[q] + 1u) & ~1u)});
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
  out.arena_elems = arena;
  out.fits = table_elems + arena <= max_elems;
  auto resolve = [&](const Ref& r) { return r.buf < 0 ? r.abs : table_elems + offset[r.buf]; };
  for (auto& p : ops) {
    SOp op = p.op;
    op.out = resolve(p.out);
    op.in1 = resolve(p.in1);
    op.in2 = resolve(p.in2);
    out.ops.push_back(op);
  }
  return out;
}

}  // namespace qtc
