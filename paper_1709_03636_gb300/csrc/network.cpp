// Circuit -> closed tensor network (Section 2), with the reverse light cone.
#include <algorithm>
#include <numeric>

#include "qtc_internal.h"

namespace qtc {

bool gate_is_diagonal(int kind) {
  return kind == QTC_GATE_Z || kind == QTC_GATE_RZ || kind == QTC_GATE_ZZ;
}

bool gate_is_channel(int kind) {
  return kind == QTC_GATE_DEPOLARIZE || kind == QTC_GATE_DEPHASE || kind == QTC_GATE_AMPDAMP;
}

namespace {

struct UnionFind {
  std::vector<int> parent;
  explicit UnionFind(int n) : parent(n) { std::iota(parent.begin(), parent.end(), 0); }
  int find(int x) {
    while (parent[x] != x) {
      parent[x] = parent[parent[x]];
      x = parent[x];
    }
    return x;
  }
  void unite(int a, int b) {
    a = find(a);
    b = find(b);
    if (a != b) parent[std::max(a, b)] = std::min(a, b);
  }
};

GateSpec spec_of(uint8_t kind, bool conj, const Gate* g) {
  GateSpec s{};
  s.kind = kind;
  s.conj = conj ? 1 : 0;
  s.slot = -1;
  s.coeff = 0.0;
  s.constant = 0.0;
  if (g && (g->kind == QTC_GATE_RX || g->kind == QTC_GATE_RZ || g->kind == QTC_GATE_ZZ)) {
    s.slot = (int16_t)g->slot;
    s.coeff = g->slot >= 0 ? g->coeff : 0.0;
    s.constant = g->constant;
  }
  if (g && gate_is_channel(g->kind)) s.constant = g->constant;  // the channel's strength
  return s;
}

GateSpec plain(uint8_t kind, bool conj) { return spec_of(kind, conj, nullptr); }

}  // namespace

// Builds <psi|M|psi> (or <x|psi>) as ket leaves, conjugated bra leaves and the
// observable.  Light cone: walking the gates backwards from the observable's
// support S, a gate that misses S commutes with the Heisenberg-picture
// operator and is dropped; so is a diagonal gate that touches S only on
// qubits where that operator is still diagonal (set D).  A kept diagonal gate
// adds its other qubits to S and D; a kept non-diagonal gate adds its qubits
// to S and removes them from D.  Only qubits of S get wires.  A noise channel
// (trace preserving: its Heisenberg-picture map fixes the identity) is
// dropped when it misses S and kept otherwise; it maps operators diagonal on
// its qubit to diagonal ones, so S and D are unchanged.  With channels the
// ket and bra sides are built in step: a channel is one tensor joining the
// ket and bra wires of its qubit (Section 2's density-matrix form).
Network build_network(const Circuit& c, const qtc_observable& obs, bool lightcone,
                      bool diag) {
  const int n = c.n;
  std::vector<char> op(n, 'I');   // 'I', 'X', 'Y', 'Z', or '0'/'1' (projector)
  bool amplitude = false, projector = false;
  std::vector<int> bits(n, 0);
  switch (obs.kind) {
    case QTC_OBS_ZZ:
      if (obs.u < 0 || obs.u >= n || obs.v < 0 || obs.v >= n || obs.u == obs.v)
        fail(QTC_ERR_INVALID, "ZZ observable qubits (%d, %d) invalid for n = %d", obs.u,
             obs.v, n);
      op[obs.u] = op[obs.v] = 'Z';
      break;
    case QTC_OBS_IDENTITY:
      if (lightcone) fail(QTC_ERR_INVALID, "the identity observable has an empty light cone");
      break;
    case QTC_OBS_PAULI:
      if (!obs.pauli) fail(QTC_ERR_INVALID, "Pauli observable without a string");
      for (int q = 0; q < n; ++q) {
        char ch = obs.pauli[q];
        if (ch != 'I' && ch != 'X' && ch != 'Y' && ch != 'Z')
          fail(QTC_ERR_INVALID, "Pauli character '%c' at qubit %d", ch, q);
        op[q] = ch;
      }
      if (lightcone && std::all_of(op.begin(), op.end(), [](char ch) { return ch == 'I'; }))
        fail(QTC_ERR_INVALID, "all-identity Pauli string has an empty light cone");
      break;
    case QTC_OBS_AMPLITUDE:
      if (lightcone) fail(QTC_ERR_INVALID, "the amplitude network has no light cone");
      if (!obs.bits) fail(QTC_ERR_INVALID, "amplitude observable without bits");
      amplitude = true;
      for (int q = 0; q < n; ++q) {
        if (obs.bits[q] > 1) fail(QTC_ERR_INVALID, "bit %d of the basis state is not 0/1", q);
        bits[q] = obs.bits[q];
      }
      break;
    case QTC_OBS_PROJECTOR: {
      if (!obs.bits) fail(QTC_ERR_INVALID, "projector observable without bits");
      projector = true;
      bool any = false;
      for (int q = 0; q < n; ++q) {
        if (obs.bits[q] > 2) fail(QTC_ERR_INVALID, "projector entry %d at qubit %d", obs.bits[q], q);
        op[q] = obs.bits[q] == 2 ? 'I' : (obs.bits[q] ? '1' : '0');
        any |= obs.bits[q] != 2;
      }
      if (lightcone && !any) fail(QTC_ERR_INVALID, "no measured qubit: empty light cone");
      break;
    }
    default:
      fail(QTC_ERR_INVALID, "unknown observable kind %d", obs.kind);
  }

  const int G = (int)c.gates.size();
  std::vector<char> keep(G, 1);
  std::vector<char> in_s(n, 1);
  if (lightcone) {
    std::vector<char> in_d(n, 0);
    for (int q = 0; q < n; ++q) {
      in_s[q] = op[q] != 'I';
      in_d[q] = op[q] == 'Z' || op[q] == '0' || op[q] == '1';  // diagonal operators
    }
    for (int gi = G - 1; gi >= 0; --gi) {
      const Gate& g = c.gates[gi];
      bool touches = false, touches_nondiag = false;
      for (int k = 0; k < g.nq; ++k) {
        touches |= in_s[g.q[k]] != 0;
        touches_nondiag |= in_s[g.q[k]] && !in_d[g.q[k]];
      }
      if (!touches || (gate_is_diagonal(g.kind) && !touches_nondiag)) {
        keep[gi] = 0;
        continue;
      }
      if (gate_is_channel(g.kind)) continue;
      for (int k = 0; k < g.nq; ++k) {
        int q = g.q[k];
        if (gate_is_diagonal(g.kind)) {
          if (!in_s[q]) in_s[q] = in_d[q] = 1;
        } else {
          in_s[q] = 1;
          in_d[q] = 0;
        }
      }
    }
  }

  // fold a first H on |0> into |+>
  std::vector<int> folded(n, -1);
  {
    std::vector<char> seen(n, 0);
    for (int gi = 0; gi < G; ++gi) {
      if (!keep[gi]) continue;
      const Gate& g = c.gates[gi];
      for (int k = 0; k < g.nq; ++k) {
        int q = g.q[k];
        if (seen[q]) continue;
        seen[q] = 1;
        if (g.kind == QTC_GATE_H) folded[q] = gi;
      }
    }
  }

  Network net;
  net.n_params = c.n_params;
  int next_label = 0;
  auto new_label = [&]() { return next_label++; };

  auto init_side = [&](bool conj, std::vector<int>& cur) {
    cur.assign(n, -1);
    for (int q = 0; q < n; ++q) {
      if (!in_s[q]) continue;
      cur[q] = new_label();
      net.leaves.push_back({plain(folded[q] >= 0 ? LK_PLUS : LK_ZERO, conj), {cur[q]}});
    }
  };
  // one unitary gate on one side (ket: conj = false, bra: conj = true)
  auto apply_gate = [&](int gi, bool conj, std::vector<int>& cur) {
    const Gate& g = c.gates[gi];
    if (g.nq == 1 && folded[g.q[0]] == gi) return;
    if (diag && gate_is_diagonal(g.kind)) {
      if (g.kind == QTC_GATE_ZZ)
        net.leaves.push_back({spec_of(LK_ZZDIAG, conj, &g), {cur[g.q[0]], cur[g.q[1]]}});
      else if (g.kind == QTC_GATE_RZ)
        net.leaves.push_back({spec_of(LK_RZDIAG, conj, &g), {cur[g.q[0]]}});
      else
        net.leaves.push_back({plain(LK_ZDIAG, conj), {cur[g.q[0]]}});
      return;
    }
    if (g.nq == 1) {
      int q = g.q[0];
      int out = new_label();
      uint8_t kind = 0;
      switch (g.kind) {
        case QTC_GATE_H: kind = LK_H; break;
        case QTC_GATE_X: kind = LK_X; break;
        case QTC_GATE_Y: kind = LK_Y; break;
        case QTC_GATE_Z: kind = LK_Z; break;
        case QTC_GATE_RX: kind = LK_RX; break;
        case QTC_GATE_RZ: kind = LK_RZ; break;
        default: fail(QTC_ERR_INVALID, "gate kind %d is not a one-qubit gate", g.kind);
      }
      net.leaves.push_back({spec_of(kind, conj, &g), {out, cur[q]}});
      cur[q] = out;
    } else if (diag && g.kind == QTC_GATE_CNOT) {
      // sparse CNOT: the control wire passes through (a hyperedge), the
      // target gets t_out = t_in xor control
      int a = g.q[0], b = g.q[1];
      int ob = new_label();
      net.leaves.push_back({plain(LK_CNOTX, conj), {ob, cur[a], cur[b]}});
      cur[b] = ob;
    } else {
      int a = g.q[0], b = g.q[1];
      int oa = new_label(), ob = new_label();
      uint8_t kind = g.kind == QTC_GATE_ZZ ? LK_ZZ : LK_CNOT;
      net.leaves.push_back({spec_of(kind, conj, &g), {oa, ob, cur[a], cur[b]}});
      cur[a] = oa;
      cur[b] = ob;
    }
  };
  auto side = [&](bool conj, std::vector<int>& cur) {
    init_side(conj, cur);
    for (int gi = 0; gi < G; ++gi)
      if (keep[gi]) apply_gate(gi, conj, cur);
  };
  bool channels = false;
  for (int gi = 0; gi < G; ++gi) channels |= keep[gi] && gate_is_channel(c.gates[gi].kind);
  if (channels && amplitude)
    fail(QTC_ERR_INVALID, "a circuit with noise channels has no amplitude network");
  if (channels && !projector) {
    // A channel that is the last operation on a qubit closed by the trace
    // (identity observable) is the identity there (trace preserving): drop
    // it, and any channels it uncovers.  (Projector networks keep it: their
    // wires close with explicit tensors, and every projector network of a
    // circuit keeps one structure.)
    for (int q = 0; q < n; ++q) {
      if (!in_s[q] || op[q] != 'I') continue;
      for (int gi = G - 1; gi >= 0; --gi) {
        if (!keep[gi]) continue;
        const Gate& g = c.gates[gi];
        bool on_q = false;
        for (int k = 0; k < g.nq; ++k) on_q |= g.q[k] == q;
        if (!on_q) continue;
        if (!gate_is_channel(g.kind)) break;
        keep[gi] = 0;
      }
    }
    channels = false;
    for (int gi = 0; gi < G; ++gi) channels |= keep[gi] && gate_is_channel(c.gates[gi].kind);
  }

  std::vector<int> ket, bra;
  if (channels) {
    // ket and bra in step; a channel joins the two wires of its qubit
    init_side(false, ket);
    init_side(true, bra);
    for (int gi = 0; gi < G; ++gi) {
      if (!keep[gi]) continue;
      const Gate& g = c.gates[gi];
      if (!gate_is_channel(g.kind)) {
        apply_gate(gi, false, ket);
        apply_gate(gi, true, bra);
        continue;
      }
      const int q = g.q[0];
      const int ko = new_label(), bo = new_label();
      const uint8_t kind = g.kind == QTC_GATE_DEPOLARIZE ? LK_DEPOL
                           : g.kind == QTC_GATE_DEPHASE  ? LK_DEPHASE
                                                         : LK_AMPDAMP;
      net.leaves.push_back({spec_of(kind, false, &g), {ko, bo, ket[q], bra[q]}});
      ket[q] = ko;
      bra[q] = bo;
    }
  } else {
    side(false, ket);
  }
  if (amplitude) {
    for (int q = 0; q < n; ++q)
      if (in_s[q]) net.leaves.push_back({plain(bits[q] ? LK_PROJ1 : LK_PROJ0, false), {ket[q]}});
  } else {
    if (!channels) side(true, bra);
    std::vector<std::pair<int, int>> unite;
    for (int q = 0; q < n; ++q) {
      if (!in_s[q]) continue;
      switch (op[q]) {
        case '0':
        case '1':
          if (diag && !channels) {
            unite.push_back({bra[q], ket[q]});
            net.leaves.push_back({plain(op[q] == '1' ? LK_PROJ1 : LK_PROJ0, false), {ket[q]}});
          } else {
            net.leaves.push_back({plain(op[q] == '1' ? LK_OBS_P1 : LK_OBS_P0, false),
                                  {bra[q], ket[q]}});
          }
          break;
        case 'I':
          // projector networks close unmeasured qubits with a tensor too, so
          // that every projector network of a circuit has one structure
          if (projector && diag && !channels) {
            unite.push_back({bra[q], ket[q]});
            net.leaves.push_back({plain(LK_ONES, false), {ket[q]}});
            break;
          }
          if (projector) {
            net.leaves.push_back({plain(LK_OBS_I, false), {bra[q], ket[q]}});
            break;
          }
          // with channels a wire is closed by an explicit identity tensor: a
          // merged label could repeat an index of a channel tensor
          if (channels)
            net.leaves.push_back({plain(LK_OBS_I, false), {bra[q], ket[q]}});
          else
            unite.push_back({bra[q], ket[q]});
          break;
        case 'Z':
          if (diag && !channels) {
            unite.push_back({bra[q], ket[q]});
            net.leaves.push_back({plain(LK_ZDIAG, false), {ket[q]}});
          } else {
            net.leaves.push_back({plain(LK_OBS_Z, false), {bra[q], ket[q]}});
          }
          break;
        case 'X':
          net.leaves.push_back({plain(LK_OBS_X, false), {bra[q], ket[q]}});
          break;
        case 'Y':
          net.leaves.push_back({plain(LK_OBS_Y, false), {bra[q], ket[q]}});
          break;
      }
    }
    UnionFind uf(next_label);
    for (auto& pr : unite) uf.unite(pr.first, pr.second);
    for (auto& leaf : net.leaves)
      for (int& l : leaf.labels) l = uf.find(l);
  }
  // compact labels in order of first appearance
  std::vector<int> remap(next_label, -1);
  int L = 0;
  for (auto& leaf : net.leaves)
    for (int& l : leaf.labels) {
      if (remap[l] < 0) remap[l] = L++;
      l = remap[l];
    }
  net.n_labels = L;
  for (auto& leaf : net.leaves) {
    if ((int)leaf.labels.size() != leaf_rank_of(leaf.spec.kind))
      fail(QTC_ERR_INVALID, "internal: leaf rank mismatch");
    for (size_t i = 0; i < leaf.labels.size(); ++i)
      for (size_t j = i + 1; j < leaf.labels.size(); ++j)
        if (leaf.labels[i] == leaf.labels[j])
          fail(QTC_ERR_UNSUPPORTED, "a leaf with a repeated index (trace) is not supported");
  }
  if (net.leaves.empty()) fail(QTC_ERR_INVALID, "the network is empty");
  return net;
}

}  // namespace qtc
