// Tile form of a global contraction (Eq. 1 with batch labels kept): which
// labels vary inside one task, how a task's footprints are copied through
// shared memory, and how its threads share the tile.  Also a host emulation
// of one tile step, used to check a lowering against the plain contraction.
#include <algorithm>
#include <cstring>
#include <string>

#include "qtc_internal.h"

namespace qtc {

namespace {

int pos_of(const std::vector<int>& v, int x) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] == x) return (int)i;
  return -1;
}

bool runs_from(const std::vector<int>& pos, GRuns& r) {
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

uint64_t apply(const GRuns& r, uint64_t idx) {
  uint64_t off = 0;
  for (int k = 0; k < r.n; ++k)
    off |= ((idx >> r.src[k]) & ((1ull << r.len[k]) - 1)) << r.dst[k];
  return off;
}

}  // namespace

bool encode_tile(GStep& g, const std::vector<int>& lc, const std::vector<int>& la,
                 const std::vector<int>& lb, bool a_table, bool b_table, size_t elem,
                 int task_terms_log2, bool direct) {
  GTileMap& t = g.tile;
  std::memset(&t, 0, sizeof t);
  std::vector<int> all(lc);
  for (int x : la)
    if (pos_of(all, x) < 0) all.push_back(x);
  for (int x : lb)
    if (pos_of(all, x) < 0) all.push_back(x);
  auto in_a = [&](int l) { return pos_of(la, l) >= 0; };
  auto in_b = [&](int l) { return pos_of(lb, l) >= 0; };
  auto in_c = [&](int l) { return pos_of(lc, l) >= 0; };
  // operands in global memory are copied through shared memory, unless the
  // tile reads them where they are (direct)
  const bool glob_a = !a_table, glob_b = !b_table;
  const bool stage_a = glob_a && !direct, stage_b = glob_b && !direct;
  const uint32_t budget = kTileBudgetBytes / (uint32_t)elem;

  std::vector<int> V;
  auto has = [&](int l) { return pos_of(V, l) >= 0; };
  auto fsize = [&](const std::vector<int>& v) {
    int fa = 0, fb = 0, fc = 0;
    for (int l : v) {
      fa += in_a(l);
      fb += in_b(l);
      fc += in_c(l);
    }
    // (read in place, the cross-warp reduction needs its own room)
    uint64_t need = (1ull << fc) + (direct ? (256ull << kTileMaxOut) : 0);
    if (stage_a) need += 1ull << fa;
    if (stage_b) need += 1ull << fb;
    return need;
  };
  auto try_add = [&](int l) {
    if (has(l)) return true;
    V.push_back(l);
    if (fsize(V) > budget) {
      V.pop_back();
      return false;
    }
    return true;
  };
  // the lowest bits of every tensor in global memory, for contiguous copies
  // (or coalesced reads)
  for (int i = 0; i < 5; ++i) {
    if (glob_a && i < (int)la.size()) V.push_back(la[i]);
    if (glob_b && i < (int)lb.size() && !has(lb[i])) V.push_back(lb[i]);
    if (i < (int)lc.size() && !has(lc[i])) V.push_back(lc[i]);
  }
  {
    std::vector<int> u;
    for (int l : V)
      if (pos_of(u, l) < 0) u.push_back(l);
    V = u;
  }
  if (fsize(V) > budget) return false;
  // summed labels, lowest in the operands first
  std::vector<int> summed;
  for (int l : all)
    if (!in_c(l)) summed.push_back(l);
  auto low = [&](int l) {
    int p = 64;
    if (in_a(l)) p = std::min(p, pos_of(la, l));
    if (in_b(l)) p = std::min(p, pos_of(lb, l));
    return p;
  };
  std::sort(summed.begin(), summed.end(), [&](int x, int y) { return low(x) < low(y); });
  int n_reg_sum = 0;
  for (int l : summed)
    if (!has(l) && n_reg_sum < kTileMaxRegSum) n_reg_sum += try_add(l);
  const size_t max_v = direct ? 8 + kTileMaxOut + kTileMaxRegSum : 24;
  // reuse: output labels an operand lacks make it be copied once per value
  // outside the tile; take them into the tile, the larger operand's first
  const double bytes_a = glob_a ? std::ldexp(1.0, (int)la.size()) : 0.0;
  const double bytes_b = glob_b ? std::ldexp(1.0, (int)lb.size()) : 0.0;
  std::vector<int> z_lab, x_lab;   // output labels not in A / not in B
  for (int l : lc) {
    if (!in_a(l)) z_lab.push_back(l);
    if (!in_b(l)) x_lab.push_back(l);
  }
  auto output_bits = [&]() {
    int n = 0;
    for (int l : V) n += in_c(l);
    return n;
  };
  const int max_out = 8 + kTileMaxOut;
  auto add_reuse = [&](const std::vector<int>& lab) {
    for (int l : lab)
      if (!has(l) && output_bits() < max_out && V.size() < max_v) try_add(l);
  };
  if (bytes_a >= bytes_b) {
    add_reuse(z_lab);
    add_reuse(x_lab);
  } else {
    add_reuse(x_lab);
    add_reuse(z_lab);
  }
  // larger tiles of output labels, lowest first, while the task stays small
  for (int l : lc) {
    if ((int)V.size() >= 13 || output_bits() >= max_out || V.size() >= max_v) break;
    if (!has(l)) try_add(l);
  }
  if (V.size() < 8 || V.size() > max_v) return false;

  // tile index order: lanes follow the larger copied operand's footprint
  // (consecutive lanes read consecutive shared-memory words), warps prefer
  // output labels, then register output labels, then register summed labels
  const std::vector<int>& lead = (glob_a && (bytes_a >= bytes_b || !glob_b)) ? la
                                 : glob_b ? lb : lc;
  std::vector<int> foot;   // V's labels in the lead tensor's bit order
  for (int l : lead)
    if (has(l)) foot.push_back(l);
  std::vector<int> order;
  for (int l : foot)
    if ((int)order.size() < 5) order.push_back(l);
  for (int l : V)
    if ((int)order.size() < 5 && pos_of(order, l) < 0) order.push_back(l);
  std::vector<int> rest;
  for (int l : V)
    if (pos_of(order, l) < 0) rest.push_back(l);
  // warps: output labels first (by C order), then summed
  std::stable_sort(rest.begin(), rest.end(), [&](int x, int y) {
    const bool cx = in_c(x), cy = in_c(y);
    if (cx != cy) return cx;
    if (cx) return pos_of(lc, x) < pos_of(lc, y);
    return low(x) < low(y);
  });
  for (int i = 0; i < 3 && i < (int)rest.size(); ++i) order.push_back(rest[i]);
  std::vector<int> reg_out, reg_sum;
  for (size_t i = 3; i < rest.size(); ++i) (in_c(rest[i]) ? reg_out : reg_sum).push_back(rest[i]);
  if ((int)reg_out.size() > kTileMaxOut || (int)reg_sum.size() > kTileMaxRegSum) return false;
  for (int l : reg_out) order.push_back(l);
  for (int l : reg_sum) order.push_back(l);
  if (order.size() != V.size()) return false;

  t.nv = (uint8_t)order.size();
  t.staged = (uint8_t)((stage_a ? 1 : 0) | (stage_b ? 2 : 0));
  t.kout = (uint8_t)reg_out.size();
  t.ns = (uint8_t)reg_sum.size();
  for (int i = 0; i < 5; ++i)
    if (!in_c(order[i])) t.sum_lane_mask |= (uint8_t)(1u << i);
  for (int i = 0; i < 3; ++i)
    if (!in_c(order[5 + i])) t.sum_warp_mask |= (uint8_t)(1u << i);

  // footprints: each tensor's tile labels in its own bit order
  auto footprint = [&](const std::vector<int>& lx) {
    std::vector<int> f;
    for (int l : lx)
      if (has(l)) f.push_back(l);
    return f;
  };
  const std::vector<int> fa = footprint(la), fb = footprint(lb), fc = footprint(lc);
  t.nfa = (uint8_t)fa.size();
  t.nfb = (uint8_t)fb.size();
  t.nfc = (uint8_t)fc.size();
  // copies move element pairs: the lowest label of each copied tensor must
  // be in its footprint first (it is, by construction, unless rank is 0)
  if (stage_a && !la.empty() && (fa.empty() || fa[0] != la[0])) return false;
  if (stage_b && !lb.empty() && (fb.empty() || fb[0] != lb[0])) return false;
  if (!lc.empty() && (fc.empty() || fc[0] != lc[0])) return false;
  std::vector<int> pa, pb, pc;
  for (int l : order) {
    pa.push_back(stage_a ? pos_of(fa, l) : pos_of(la, l));
    pb.push_back(stage_b ? pos_of(fb, l) : pos_of(lb, l));
    pc.push_back(pos_of(fc, l));
  }
  bool ok = runs_from(pa, t.tfa) && runs_from(pb, t.tfb) && runs_from(pc, t.tfc);
  std::vector<int> qa_, qb_, qc_;
  for (int l : fa) qa_.push_back(pos_of(la, l));
  for (int l : fb) qb_.push_back(pos_of(lb, l));
  for (int l : fc) qc_.push_back(pos_of(lc, l));
  ok = ok && runs_from(qa_, t.ffa) && runs_from(qb_, t.ffb) && runs_from(qc_, t.ffc);
  // outer labels
  std::vector<int> outer_c, outer_y;
  for (int l : lc)
    if (!has(l)) outer_c.push_back(l);
  for (int l : summed)
    if (!has(l)) outer_y.push_back(l);
  t.no = (uint8_t)outer_c.size();
  t.nq = (uint8_t)outer_y.size();
  std::vector<int> oa_, ob_, oc_, ya_, yb_;
  for (int l : outer_c) {
    oa_.push_back(pos_of(la, l));
    ob_.push_back(pos_of(lb, l));
    oc_.push_back(pos_of(lc, l));
  }
  for (int l : outer_y) {
    ya_.push_back(pos_of(la, l));
    yb_.push_back(pos_of(lb, l));
  }
  ok = ok && runs_from(oa_, t.oa) && runs_from(ob_, t.ob) && runs_from(oc_, t.oc) &&
       runs_from(ya_, t.qa) && runs_from(yb_, t.qb);
  if (!ok) return false;
  if (t.no > 31 || t.nq > 31) return false;

  // tasks: one per outer output value, all outer summed values inside it;
  // with the whole output in the tile, the outer summed values are cut
  // into chunks of about 2^task_terms_log2 multiply-adds
  const uint64_t nq = 1ull << t.nq;
  if (t.no == 0 && t.nq > 0) {
    uint64_t per = std::max<uint64_t>(1, (1ull << task_terms_log2) >> t.nv);
    per = std::min(per, nq);
    t.q_per_chunk = (uint32_t)per;
    g.n_chunks = (uint32_t)((nq + per - 1) / per);
    if (g.n_chunks > 1) g.flags |= GSF_SPLIT;
    t.o_per_chunk = 1;
  } else {
    // several outer output values per task when one is little work
    t.q_per_chunk = (uint32_t)nq;
    const int per_o = t.nv + t.nq;
    uint64_t per = per_o >= task_terms_log2 ? 1 : (1ull << (task_terms_log2 - per_o));
    per = std::min<uint64_t>(per, 1ull << t.no);
    t.o_per_chunk = (uint32_t)per;
    g.n_chunks = (uint32_t)(((1ull << t.no) + per - 1) / per);
  }
  if (g.flags & GSF_LEAFGRAD) {
    // dS/dleaf reduced against the leaf derivative by the last chunk
    if (t.no != 0) return false;
    g.flags |= GSF_SPLIT;
  }
  g.chunk = t.q_per_chunk;
  g.flags |= GSF_TILE;
  return true;
}

size_t tile_region_bytes(const GStep& g, size_t elem) {
  const GTileMap& t = g.tile;
  // [A footprint | B footprint] (or, for the cross-warp reduction after the
  // contraction, every thread's accumulators: 256 << kout elements), then the
  // C footprint, then the register-summed offsets (two words each); each
  // footprint of complex64 is at least one 16-byte pair
  const size_t min_fp = elem == 8 ? 2 : 1;
  size_t ab = 0;
  if (t.staged & 1) ab += std::max(min_fp, (size_t)1 << t.nfa);
  if (t.staged & 2) ab += std::max(min_fp, (size_t)1 << t.nfb);
  if (t.sum_warp_mask) ab = std::max(ab, (size_t)256 << t.kout);
  const size_t c = std::max(min_fp, (size_t)1 << t.nfc);
  return (((ab + c) * elem + 15) & ~size_t(15)) + ((size_t)8 << t.ns);
}

// Host emulation of a tile step: the kernel's copies, thread decomposition
// and reductions on explicit arrays, checked against the plain sum over the
// step's row/summed bit maps.  Returns the largest absolute difference.
double emulate_tile_step(const GStep& g, uint64_t seed) {
  const GTileMap& t = g.tile;
  const uint64_t ra = (apply(g.ca, (1ull << g.rc) - 1) | apply(g.ya, (1ull << g.ry) - 1)) + 1;
  const uint64_t rb = (apply(g.cb, (1ull << g.rc) - 1) | apply(g.yb, (1ull << g.ry) - 1)) + 1;
  SplitMix64 rng(seed);
  auto draw = [&]() { return std::complex<double>((double)(rng.next() >> 11) * 0x1p-53 - 0.5,
                                                  (double)(rng.next() >> 11) * 0x1p-53 - 0.5); };
  std::vector<std::complex<double>> A(ra), B(rb), C(1ull << g.rc, 0.0), R(1ull << g.rc, 0.0);
  for (auto& x : A) x = draw();
  for (auto& x : B) x = draw();
  // plain: C[c] = sum_y A[ca(c) | ya(y)] B[cb(c) | yb(y)]
  for (uint64_t c = 0; c < (1ull << g.rc); ++c)
    for (uint64_t y = 0; y < (1ull << g.ry); ++y)
      R[c] += A[apply(g.ca, c) | apply(g.ya, y)] * B[apply(g.cb, c) | apply(g.yb, y)];
  // tile form, chunk by chunk
  const bool sa = (t.staged & 1) != 0, sb = (t.staged & 2) != 0;
  const uint64_t nq = 1ull << t.nq;
  std::vector<std::complex<double>> partial;
  const bool split = (g.flags & GSF_SPLIT) != 0;
  if (split) partial.assign((size_t)g.n_chunks << t.nfc, 0.0);
  for (uint64_t task_o = 0; task_o < (split ? 1 : (1ull << t.no)); ++task_o)
  for (uint32_t chunk = 0; chunk < (split ? g.n_chunks : 1); ++chunk) {
    const uint64_t o = task_o;
    const uint64_t q0 = split ? (uint64_t)chunk * t.q_per_chunk : 0;
    const uint64_t q1 = split ? std::min<uint64_t>(q0 + t.q_per_chunk, nq) : nq;
    std::vector<std::complex<double>> Cs(1ull << t.nfc, 0.0);
    // per thread (lane, warp) and register output k: accumulators
    std::vector<std::complex<double>> acc((size_t)256 << t.kout, 0.0);
    for (uint64_t q = q0; q < q1; ++q) {
      const uint64_t abase = apply(t.oa, o) | apply(t.qa, q);
      const uint64_t bbase = apply(t.ob, o) | apply(t.qb, q);
      std::vector<std::complex<double>> As, Bs;
      if (sa) {
        As.resize(1ull << t.nfa);
        for (uint64_t j = 0; j < As.size(); ++j) As[j] = A[abase | apply(t.ffa, j)];
      }
      if (sb) {
        Bs.resize(1ull << t.nfb);
        for (uint64_t j = 0; j < Bs.size(); ++j) Bs[j] = B[bbase | apply(t.ffb, j)];
      }
      for (uint32_t th = 0; th < 256; ++th)
        for (uint32_t k = 0; k < (1u << t.kout); ++k)
          for (uint32_t s = 0; s < (1u << t.ns); ++s) {
            const uint64_t ti = th | ((uint64_t)k << 8) | ((uint64_t)s << (8 + t.kout));
            const std::complex<double> a = sa ? As[apply(t.tfa, ti)] : A[abase | apply(t.tfa, ti)];
            const std::complex<double> b = sb ? Bs[apply(t.tfb, ti)] : B[bbase | apply(t.tfb, ti)];
            acc[((size_t)th << t.kout) | k] += a * b;
          }
    }
    // lane and warp reductions, owners write the C tile
    for (uint32_t th = 0; th < 256; ++th) {
      const uint32_t lane = th & 31, warp = th >> 5;
      if ((lane & t.sum_lane_mask) || (warp & t.sum_warp_mask)) continue;
      for (uint32_t k = 0; k < (1u << t.kout); ++k) {
        std::complex<double> sum = 0.0;
        for (uint32_t l2 = 0; l2 < 32; ++l2)
          for (uint32_t w2 = 0; w2 < 8; ++w2)
            if ((l2 & ~t.sum_lane_mask) == lane && (w2 & ~t.sum_warp_mask) == warp)
              sum += acc[((size_t)(l2 | (w2 << 5)) << t.kout) | k];
        const uint64_t ti = th | ((uint64_t)k << 8);
        Cs[apply(t.tfc, ti)] = sum;
      }
    }
    const uint64_t cbase = apply(t.oc, o);
    if (split) {
      for (uint64_t j = 0; j < Cs.size(); ++j) partial[((size_t)chunk << t.nfc) + j] = Cs[j];
    } else {
      for (uint64_t j = 0; j < Cs.size(); ++j) C[cbase | apply(t.ffc, j)] = Cs[j];
    }
  }
  if (split)
    for (uint64_t j = 0; j < (1ull << t.nfc); ++j) {
      std::complex<double> sum = 0.0;
      for (uint32_t k = 0; k < g.n_chunks; ++k) sum += partial[((size_t)k << t.nfc) + j];
      C[apply(t.ffc, j)] = sum;
    }
  double err = 0;
  for (uint64_t c = 0; c < C.size(); ++c) err = std::max(err, std::abs(C[c] - R[c]));
  return err;
}

// Host emulation of a GSF_ROWS step: per chunk the kernel's row tables, and
// per group of four rows only the group's distinct operand elements (A by
// ia(k), B by ib(k)), against the plain sum over every output's own bit maps.
double emulate_rows_step(const GStep& g, uint64_t seed) {
  const uint64_t ra = (apply(g.ca, (1ull << g.rc) - 1) | apply(g.ya, (1ull << g.ry) - 1)) + 1;
  const uint64_t rb = (apply(g.cb, (1ull << g.rc) - 1) | apply(g.yb, (1ull << g.ry) - 1)) + 1;
  SplitMix64 rng(seed);
  auto draw = [&]() { return std::complex<double>((double)(rng.next() >> 11) * 0x1p-53 - 0.5,
                                                  (double)(rng.next() >> 11) * 0x1p-53 - 0.5); };
  std::vector<std::complex<double>> A(ra), B(rb), C(1ull << g.rc, 0.0), R(1ull << g.rc, 0.0);
  std::vector<char> written(1ull << g.rc, 0);
  for (auto& x : A) x = draw();
  for (auto& x : B) x = draw();
  const uint64_t ny = 1ull << g.ry;
  for (uint64_t c = 0; c < (1ull << g.rc); ++c)
    for (uint64_t y = 0; y < ny; ++y)
      R[c] += A[apply(g.ca, c) | apply(g.ya, y)] * B[apply(g.cb, c) | apply(g.yb, y)];
  const uint64_t rowlen = kGRow;
  for (uint32_t chunk = 0; chunk < g.n_chunks; ++chunk) {
    const uint64_t r0 = (uint64_t)chunk * g.chunk;
    std::vector<uint64_t> rowa(g.chunk), rowb(g.chunk), rowc(g.chunk);
    for (uint32_t r = 0; r < g.chunk; ++r) {
      const uint64_t o = apply(g.rows, r0 + r);
      rowa[r] = apply(g.ca, o * rowlen);
      rowb[r] = apply(g.cb, o * rowlen);
      rowc[r] = o * rowlen;
    }
    // a group's distinct elements: A by the counter bits it holds (the row
    // with the others clear), B likewise
    const bool fixed = g.share == GRS_FIXA || g.share == GRS_FIXB;
    const int ng = 1 << (fixed ? grs_fix_bits((uint32_t)ny) : 2);
    const int ma = g.share == GRS_ZX ? 2 : g.share == GRS_ZZ ? 0
                   : g.share == GRS_FIXA ? 0 : ng - 1;   // counter bits A varies with
    const int mb = g.share == GRS_ZX ? 1 : g.share == GRS_XX ? 0
                   : g.share == GRS_FIXB ? 0 : ng - 1;
    for (uint32_t r = 0; r < g.chunk; r += ng)
      for (uint64_t tid = 0; tid < rowlen; ++tid) {
        const uint64_t a_lo = apply(g.ca, tid), b_lo = apply(g.cb, tid);
        for (int k = 0; k < ng; ++k) {
          const uint64_t oa = rowa[r + (k & ma)] | a_lo;
          const uint64_t ob = rowb[r + (k & mb)] | b_lo;
          std::complex<double> acc = 0.0;
          for (uint64_t y = 0; y < ny; ++y) acc += A[oa | apply(g.ya, y)] * B[ob | apply(g.yb, y)];
          C[rowc[r + k] + tid] = acc;
          written[rowc[r + k] + tid] = 1;
        }
      }
  }
  double err = 0;
  for (uint64_t c = 0; c < C.size(); ++c)
    err = std::max(err, written[c] ? std::abs(C[c] - R[c]) : 1e30);
  return err;
}

}  // namespace qtc
