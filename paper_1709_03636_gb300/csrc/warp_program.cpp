// Warp programs for networks run one per warp: the lowered shared-memory ops
// of one network (pairwise contractions of Eq. 1 with batch indices, the
// adjoint sweep and the leaf-gradient dots) become warp steps.
//
// Each op first gets its bit maps expanded into per-lane offset tables (a
// WOp), and a leaf-gradient dot that reads the tensor the previous op wrote
// is fused into that op.  Then the ops are list-scheduled: an op whose
// output has at most 32 elements and whose sum has at most two terms takes
// an aligned group of 2^rc lanes in the earliest step after every op it
// depends on, where dependences are read-after-write, write-after-read and
// write-after-write on individual arena elements (the arena reuses buffers).
// Larger ops get a step of their own (solo).  The step count, not the op
// count, then bounds the network's latency on the warp.
#include <algorithm>
#include <cstring>

#include "qtc_internal.h"

namespace qtc {

namespace {

uint16_t deposit(const uint8_t* pos, int first, int count, uint32_t idx) {
  uint32_t off = 0;
  for (int i = 0; i < count; ++i)
    if (((idx >> i) & 1u) && pos[first + i] != kAbsent) off |= 1u << pos[first + i];
  return (uint16_t)off;
}

WOp expand(const SOp& op) {
  WOp w{};
  w.code = op.code;
  w.rc = op.rc;
  w.ry = op.ry;
  w.out = (uint16_t)op.out;
  w.in1 = (uint16_t)op.in1;
  w.in2 = (uint16_t)op.in2;
  w.slot = (uint16_t)op.out;
  if (op.code == SOP_CONTRACT) {
    const int lo = std::min<int>(op.rc, 5), hi = std::max<int>(op.rc - 5, 0);
    for (uint32_t c = 0; c < 32; ++c) {
      w.a_lo[c] = deposit(op.p1, 0, lo, c);
      w.b_lo[c] = deposit(op.p2, 0, lo, c);
    }
    for (uint32_t j = 0; j < 64; ++j) {
      w.a_hi[j] = deposit(op.p1, 5, hi, j);
      w.b_hi[j] = deposit(op.p2, 5, hi, j);
    }
    for (uint32_t y = 0; y < 16; ++y) {
      w.ya[y] = deposit(op.y1, 0, std::min<int>(op.ry, 4), y);
      w.yb[y] = deposit(op.y2, 0, std::min<int>(op.ry, 4), y);
      w.ya_hi[y] = deposit(op.y1, 4, std::max<int>(op.ry - 4, 0), y);
      w.yb_hi[y] = deposit(op.y2, 4, std::max<int>(op.ry - 4, 0), y);
    }
  }
  return w;
}

struct Access {
  std::vector<uint32_t> reads, writes;   // arena element indices
};

// Arena elements an op reads and writes (gate-table operands are read-only).
Access accesses(const WOp& w, uint32_t table_elems) {
  Access acc;
  auto arena = [&](uint32_t base, uint32_t rel, std::vector<uint32_t>& v) {
    if (base >= table_elems) v.push_back(base - table_elems + rel);
  };
  const uint32_t nout = 1u << w.rc;
  switch (w.code) {
    case SOP_CONTRACT:
      for (uint32_t c = 0; c < nout; ++c) {
        const uint32_t oa = w.a_lo[c & 31] | w.a_hi[c >> 5], ob = w.b_lo[c & 31] | w.b_hi[c >> 5];
        for (uint32_t y = 0; y < (1u << w.ry); ++y) {
          arena(w.in1, oa | w.ya[y & 15] | w.ya_hi[y >> 4], acc.reads);
          arena(w.in2, ob | w.yb[y & 15] | w.yb_hi[y >> 4], acc.reads);
        }
        arena(w.out, c, acc.writes);
      }
      break;
    case SOP_LEAFGRAD:
      for (uint32_t c = 0; c < nout; ++c) {
        arena(w.in1, c, acc.reads);
        arena(w.in2, c, acc.reads);
      }
      break;
    case SOP_RESULT:
      arena(w.in1, 0, acc.reads);
      break;
    case SOP_SEED:
      arena(w.out, 0, acc.writes);
      break;
    default:
      break;
  }
  return acc;
}

// Lane offsets are team relative: the warp's own gate-table copy first, then
// its arena (the same numbering as the shared-memory ops).
uint16_t lane_operand(uint32_t off, uint32_t) { return (uint16_t)off; }

struct Slotted {
  uint32_t mask = 0;   // lanes in use
  bool solo = false;
  WStep step{};
};

}  // namespace

void build_warp_steps(const std::vector<SOp>& ops, uint32_t table_elems, uint32_t arena_elems,
                      std::vector<WStep>& out) {
  // expand, fusing LEAFGRAD into the CONTRACT that produces its operand
  std::vector<WOp> wops;
  for (const SOp& op : ops) {
    if (op.code == SOP_LEAFGRAD && !wops.empty()) {
      WOp& prev = wops.back();
      if (prev.code == SOP_CONTRACT && !(prev.flags & WOPF_LEAFGRAD) && prev.out == op.in1 &&
          prev.rc == op.rc) {
        prev.flags |= WOPF_LEAFGRAD;
        prev.der = (uint16_t)op.in2;
        prev.slot = (uint16_t)op.out;
        continue;
      }
    }
    wops.push_back(expand(op));
  }

  std::vector<int> last_read(arena_elems + 1, -1), last_write(arena_elems + 1, -1);
  std::vector<Slotted> steps;
  for (const WOp& w : wops) {
    const Access acc = accesses(w, table_elems);
    int earliest = 0;
    for (uint32_t e : acc.reads) earliest = std::max(earliest, last_write[e] + 1);
    for (uint32_t e : acc.writes)
      earliest = std::max({earliest, last_read[e] + 1, last_write[e] + 1});
    // 2^ry summed terms (ry = 2..4): 2^(ry-1) lanes per output, two terms each,
    // added by shuffles
    const bool paired = w.code == SOP_CONTRACT && w.ry >= 2 && w.ry <= 4 &&
                        w.rc + w.ry - 1 <= 5;
    const bool bundled =
        (w.code == SOP_CONTRACT && w.rc <= 5 && w.ry <= 1) || paired ||
        (w.code == SOP_LEAFGRAD && w.rc <= 5) || w.code == SOP_RESULT || w.code == SOP_SEED;
    const uint32_t gw = paired ? (uint32_t)(w.rc + w.ry - 1)
                               : (w.code == SOP_CONTRACT || w.code == SOP_LEAFGRAD) ? w.rc : 0;
    const uint32_t width = 1u << gw;
    const uint32_t group = width == 32 ? 0xFFFFFFFFu : ((1u << width) - 1u);
    int at = -1;
    uint32_t pos = 0;
    for (int s = earliest; s < (int)steps.size() && at < 0; ++s) {
      if (steps[s].solo) continue;
      if (!bundled) {
        if (steps[s].mask == 0) at = s;
        continue;
      }
      for (uint32_t p = 0; p < 32; p += width)
        if (!(steps[s].mask & (group << p))) {
          at = s;
          pos = p;
          break;
        }
    }
    if (at < 0) {
      at = (int)steps.size();
      steps.emplace_back();
    }
    Slotted& st = steps[at];
    if (!bundled) {
      st.solo = true;
      st.mask = 0xFFFFFFFFu;
      st.step.solo = 1;
      st.step.op = w;
    } else if (paired) {
      st.mask |= group << pos;
      auto yoff = [](const uint16_t* lo, const uint16_t* hi, uint32_t y) {
        return (uint32_t)(lo[y & 15] | hi[y >> 4]);
      };
      st.step.pad[0] = (uint8_t)std::max<uint32_t>(st.step.pad[0], w.ry - 1u);
      for (uint32_t i = 0; i < width; ++i) {
        WLane& l = st.step.lane[pos + i];
        const uint32_t c = i & ((1u << w.rc) - 1u), yh = i >> w.rc;  // y = 2 yh + ylo
        const bool first = yh == 0;
        const bool leaf = first && (w.flags & WOPF_LEAFGRAD);
        l.gw = (uint8_t)(gw | (uint32_t)w.rc << 3 | (uint32_t)(w.ry - 1) << 6);
        l.slot = leaf ? (uint8_t)w.slot : (uint8_t)0;
        l.kind = WL_CONTRACT;
        l.flags = (uint8_t)(WLF_Y1 | (first ? WLF_STORE : 0) | (leaf ? WLF_LG_MUL : 0));
        l.c_off = (uint16_t)(w.out + c);
        l.a_off = (uint16_t)(lane_operand(w.in1, table_elems) +
                             (w.a_lo[c] | yoff(w.ya, w.ya_hi, 2 * yh)));
        l.b_off = (uint16_t)(lane_operand(w.in2, table_elems) +
                             (w.b_lo[c] | yoff(w.yb, w.yb_hi, 2 * yh)));
        l.ya1 = (uint16_t)yoff(w.ya, w.ya_hi, 1);
        l.yb1 = (uint16_t)yoff(w.yb, w.yb_hi, 1);
        if (leaf) {
          l.der_off = (uint16_t)(w.der + c);
          st.step.rounds = (uint8_t)(kWHasLeafGrad |
                                     std::max<uint32_t>(st.step.rounds & 0x7Fu, gw));
        }
      }
    } else {
      st.mask |= group << pos;
      for (uint32_t c = 0; c < width; ++c) {
        WLane& l = st.step.lane[pos + c];
        l.gw = (uint8_t)gw;
        // the parameter slot of a leaf-gradient lane; 0 for the others
        const bool leaf = (w.code == SOP_CONTRACT && (w.flags & WOPF_LEAFGRAD)) ||
                          w.code == SOP_LEAFGRAD;
        l.slot = leaf ? (uint8_t)w.slot : (uint8_t)0;
        if (w.code == SOP_CONTRACT) {
          l.kind = WL_CONTRACT;
          l.flags = WLF_STORE;
          l.c_off = (uint16_t)(w.out + c);
          l.a_off = (uint16_t)(lane_operand(w.in1, table_elems) + w.a_lo[c]);
          l.b_off = (uint16_t)(lane_operand(w.in2, table_elems) + w.b_lo[c]);
          if (w.ry == 1) {
            l.flags |= WLF_Y1;
            l.ya1 = w.ya[1];
            l.yb1 = w.yb[1];
          }
          if (w.flags & WOPF_LEAFGRAD) {
            l.flags |= WLF_LG_MUL;
            l.der_off = (uint16_t)(w.der + c);
          }
        } else if (w.code == SOP_LEAFGRAD) {
          l.kind = WL_CONTRACT;
          l.flags = WLF_LG_ADD;
          l.a_off = (uint16_t)(lane_operand(w.in1, table_elems) + c);
          l.b_off = (uint16_t)(lane_operand(w.in2, table_elems) + c);
        } else if (w.code == SOP_RESULT) {
          l.kind = WL_RESULT;
          l.a_off = lane_operand(w.in1, table_elems);
        } else {
          l.kind = WL_SEED;
          l.flags = WLF_STORE;
          l.c_off = (uint16_t)w.out;
        }
        if (l.flags & (WLF_LG_MUL | WLF_LG_ADD))
          st.step.rounds = (uint8_t)(kWHasLeafGrad |
                                     std::max<uint32_t>(st.step.rounds & 0x7Fu, gw));
      }
    }
    for (uint32_t e : acc.reads) last_read[e] = std::max(last_read[e], at);
    for (uint32_t e : acc.writes) last_write[e] = at;
  }
  for (Slotted& st : steps) {
    if (!st.solo)
      for (int l = 0; l < 32; ++l)
        if (!(st.mask & (1u << l))) {
          // idle lanes read table element 0 and write nothing
          st.step.lane[l] = WLane{};
        }
    out.push_back(st.step);
  }
}

}  // namespace qtc

namespace qtc {

// Every shared-memory access a warp program can make, checked on the host
// against the team's region (gate-table copy + arena, `team_elems`
// elements), and every shuffle and gradient slot against its bounds; throws
// on the first violation.
void validate_warp_steps(const WStep* steps, size_t n, uint32_t team_elems, int n_params) {
  auto need = [&](bool ok, size_t k, int lane, const char* what) {
    if (!ok) fail(QTC_ERR_INVALID, "internal: warp step %zu lane %d: %s", k, lane, what);
  };
  for (size_t k = 0; k < n; ++k) {
    const WStep& st = steps[k];
    if (st.solo) {
      const WOp& w = st.op;
      const uint32_t nout = 1u << w.rc, ny = 1u << w.ry;
      need(w.rc <= kWarpMaxRank && w.ry <= kWarpMaxSummed, k, -1, "op shape");
      if (w.code == SOP_CONTRACT) {
        uint32_t ma = 0, mb = 0;
        for (uint32_t c = 0; c < nout; ++c) {
          ma = std::max<uint32_t>(ma, w.a_lo[c & 31] | w.a_hi[c >> 5]);
          mb = std::max<uint32_t>(mb, w.b_lo[c & 31] | w.b_hi[c >> 5]);
        }
        uint32_t ya = 0, yb = 0;
        for (uint32_t y = 0; y < ny; ++y) {
          ya = std::max<uint32_t>(ya, w.ya[y & 15] | w.ya_hi[y >> 4]);
          yb = std::max<uint32_t>(yb, w.yb[y & 15] | w.yb_hi[y >> 4]);
        }
        need((size_t)w.in1 + (ma | ya) < team_elems, k, -1, "first operand");
        need((size_t)w.in2 + (mb | yb) < team_elems, k, -1, "second operand");
        need((size_t)w.out + nout <= team_elems, k, -1, "output");
        if (w.flags & WOPF_LEAFGRAD) {
          need((size_t)w.der + nout <= team_elems, k, -1, "leaf derivative");
          need(w.slot < n_params, k, -1, "gradient slot");
        }
      } else if (w.code == SOP_LEAFGRAD) {
        need((size_t)w.in1 + nout <= team_elems && (size_t)w.in2 + nout <= team_elems, k, -1,
             "leaf-gradient operands");
        need(w.slot < n_params, k, -1, "gradient slot");
      } else if (w.code == SOP_RESULT) {
        need(w.in1 < team_elems, k, -1, "result operand");
      } else if (w.code == SOP_SEED) {
        need(w.out < team_elems, k, -1, "seed");
      }
      continue;
    }
    need((st.rounds & 0x7Fu) <= 5 && st.pad[0] <= 3, k, -1, "step rounds");
    for (int l = 0; l < 32; ++l) {
      const WLane& L = st.lane[l];
      const uint32_t gw = L.gw & 7u, pd = (L.gw >> 3) & 7u, pr = L.gw >> 6;
      need(gw <= 5 && pd + pr <= 5 && pr <= st.pad[0], k, l, "lane group");
      need(L.a_off < team_elems && L.b_off < team_elems, k, l, "operands");
      if (L.flags & WLF_Y1)
        need((size_t)L.a_off + L.ya1 < team_elems && (size_t)L.b_off + L.yb1 < team_elems, k,
             l, "second term");
      if (L.flags & WLF_STORE) need(L.c_off < team_elems, k, l, "output");
      if (L.flags & WLF_LG_MUL) need(L.der_off < team_elems, k, l, "leaf derivative");
      if (L.flags & (WLF_LG_MUL | WLF_LG_ADD)) need(L.slot < n_params, k, l, "gradient slot");
    }
  }
}

}  // namespace qtc
