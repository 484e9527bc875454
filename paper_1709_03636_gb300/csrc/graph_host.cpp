// Host side of the graph executor: per-network units -> waves of tasks.
#include <algorithm>
#include <cmath>
#include <queue>
#include <tuple>

#include "qtc_internal.h"

namespace qtc {

namespace {

uint32_t rebase32(uint64_t base, uint32_t local) {
  const uint64_t v = base + local;
  if (v >> 32) fail(QTC_ERR_ARENA, "a wave's work buffer exceeds 2^32 elements");
  return (uint32_t)v;
}

uint64_t runs_max(const GRuns& r, uint32_t bits);

// Expected time of one task of a unit on one team (ns): a chunk task moves
// its share of the step's operand and output bytes at the rate measured for
// its class of step (by summed bits; split reductions apart) divided over
// the resident teams, plus a fixed cost per task.
double task_time_estimate(const GUnit& u, size_t elem, int teams) {
  if (u.kind == GT_SMEM) return 30000.0;
  if (u.kind == GT_TC) return 5000.0;
  const GStep& st = u.step;
  const double a = (st.flags & GSF_A_TABLE)
                       ? 0.0
                       : (double)((runs_max(st.ca, st.rc) | runs_max(st.ya, st.ry)) + 1);
  const double b = (st.flags & GSF_B_TABLE)
                       ? 0.0
                       : (double)((runs_max(st.cb, st.rc) | runs_max(st.yb, st.ry)) + 1);
  const double c = (st.flags & GSF_LEAFGRAD) ? 0.0 : std::ldexp(1.0, st.rc);
  // measured per class (p=3 n=60, instrumented copy), bytes per ns over all teams
  static const double kRate[6] = {7500, 4700, 3000, 2300, 2000, 2300};
  static const double kRateFixed[3] = {8700, 7900, 4700};   // short sums, shared rows
  static const double kRateShared[6] = {0, 0, 0, 2700, 2100, 2700};   // long sums, shared rows
  const int ry = std::min<int>(st.ry, 5);
  double rate = kRate[ry];
  if (st.flags & GSF_SPLIT) rate = 3900.0;
  else if ((st.flags & GSF_ROWS) && (st.share == GRS_FIXA || st.share == GRS_FIXB) && ry <= 2)
    rate = kRateFixed[ry];
  else if ((st.flags & GSF_ROWS) && ry >= 3) rate = kRateShared[ry];
  const double bytes = (double)elem * (a + b + c) / std::max<uint32_t>(st.n_chunks, 1);
  return 1000.0 + bytes * teams / rate;
}

WaveHost assemble_wave(const std::vector<int>& nets, const std::vector<NetGraph>& graphs,
                       size_t elem, int teams) {
  WaveHost w;
  std::vector<std::vector<uint32_t>> ctr(nets.size()), arrive(nets.size());
  std::vector<uint64_t> base(nets.size());
  std::vector<size_t> uoff(nets.size() + 1, 0);
  uint32_t next_ctr = 0;
  uint64_t gsize = 0;
  for (size_t k = 0; k < nets.size(); ++k) {
    const NetGraph& g = graphs[nets[k]];
    base[k] = gsize;
    gsize += (g.global_elems + 63) & ~uint64_t(63);
    uoff[k + 1] = uoff[k] + g.units.size();
    ctr[k].resize(g.units.size());
    arrive[k].assign(g.units.size(), 0xFFFFFFFFu);
    for (size_t u = 0; u < g.units.size(); ++u) {
      ctr[k][u] = next_ctr++;
      if (g.units[u].kind == GT_CHUNK && (g.units[u].step.flags & GSF_SPLIT))
        arrive[k][u] = next_ctr++;
    }
  }
  w.global_elems = gsize;
  w.n_counters = next_ctr;
  // Each unit's records (ops, step, waits) and the template of its tasks, in
  // dependency-depth order.
  const size_t U = uoff.back();
  std::vector<GTask> tmpl(U);
  std::vector<uint32_t> n_tasks(U, 1);
  std::vector<double> dur(U), rank(U, 0.0);
  std::vector<int> depth(U);
  std::vector<std::tuple<int, int, int>> order;
  for (size_t k = 0; k < nets.size(); ++k)
    for (size_t u = 0; u < graphs[nets[k]].units.size(); ++u)
      order.emplace_back(graphs[nets[k]].units[u].depth, (int)k, (int)u);
  std::sort(order.begin(), order.end());
  for (const auto& item : order) {
    const int k = std::get<1>(item), ui = std::get<2>(item);
    const size_t gid = uoff[k] + ui;
    const NetGraph& g = graphs[nets[k]];
    const GUnit& u = g.units[ui];
    depth[gid] = u.depth;
    dur[gid] = task_time_estimate(u, elem, teams);
    const uint32_t wait_begin = (uint32_t)w.waits.size();
    for (int d : u.deps) w.waits.push_back({ctr[k][d], g.units[d].target});
    GTask t{};
    t.net = (uint32_t)nets[k];
    t.wait_begin = wait_begin;
    t.wait_count = (uint32_t)u.deps.size();
    t.signal = 0xFFFFFFFFu;
    if (u.kind == GT_SMEM) {
      t.kind = GT_SMEM;
      t.a = (uint32_t)w.ops.size();
      t.b = (uint32_t)u.ops.size();
      t.signal = ctr[k][ui];
      for (SOp op : u.ops) {
        if (op.flags & SOPF_OUT_GLOBAL) op.out = rebase32(base[k], op.out);
        if (op.flags & SOPF_IN1_GLOBAL) op.in1 = rebase32(base[k], op.in1);
        if (op.flags & SOPF_IN2_GLOBAL) op.in2 = rebase32(base[k], op.in2);
        w.ops.push_back(op);
      }
    } else if (u.kind == GT_TC) {
      TStep ts = u.tstep;
      ts.net = (uint32_t)nets[k];
      ts.done_ctr = ctr[k][ui];
      ts.c_off = rebase32(base[k], ts.c_off);
      ts.a_off = rebase32(base[k], ts.a_off);
      ts.b_off = rebase32(base[k], ts.b_off);
      t.kind = GT_TC;
      t.a = (uint32_t)w.tsteps.size();
      n_tasks[gid] = u.target;
      w.tsteps.push_back(ts);
    } else {
      GStep st = u.step;
      st.net = (uint32_t)nets[k];
      st.done_ctr = ctr[k][ui];
      st.arrive_ctr = arrive[k][ui];
      if (!(st.flags & GSF_LEAFGRAD)) st.c_off = rebase32(base[k], st.c_off);
      if (!(st.flags & GSF_A_TABLE)) st.a_off = rebase32(base[k], st.a_off);
      if (!(st.flags & GSF_B_TABLE)) st.b_off = rebase32(base[k], st.b_off);
      if (st.flags & GSF_SPLIT) st.partial_off = rebase32(base[k], st.partial_off);
      t.kind = GT_CHUNK;
      t.a = (uint32_t)w.steps.size();
      n_tasks[gid] = st.n_chunks;
      w.steps.push_back(st);
    }
    tmpl[gid] = t;
  }
  // Queue order from a list-scheduling run on the host: `teams` teams take
  // tasks as they become free, each the next task of the ready unit (all its
  // producers complete) with the longest chain of expected task times to the
  // end of its network; tasks enter the queue in the order they start.
  // Every task then comes after the tasks it waits for (no team can wait on
  // a task behind it in the queue), and teams that take tasks in this order
  // seldom wait when the estimates hold.
  std::vector<std::vector<int>> succ(U);
  std::vector<int> n_deps(U, 0);
  for (size_t k = 0; k < nets.size(); ++k) {
    const NetGraph& g = graphs[nets[k]];
    for (size_t u = 0; u < g.units.size(); ++u) {
      n_deps[uoff[k] + u] = (int)g.units[u].deps.size();
      for (int d : g.units[u].deps) succ[uoff[k] + d].push_back((int)(uoff[k] + u));
    }
  }
  std::vector<int> by_depth(U);
  for (size_t i = 0; i < U; ++i) by_depth[i] = (int)i;
  std::stable_sort(by_depth.begin(), by_depth.end(),
                   [&](int a, int b) { return depth[a] > depth[b]; });
  for (int gid : by_depth) {
    double tail = 0.0;
    for (int s : succ[gid]) tail = std::max(tail, rank[s]);
    rank[gid] = dur[gid] + tail;
  }
  auto lower = [&](int a, int b) { return rank[a] < rank[b] || (rank[a] == rank[b] && a > b); };
  std::priority_queue<int, std::vector<int>, decltype(lower)> ready(lower);
  using Event = std::pair<double, int>;
  std::priority_queue<Event, std::vector<Event>, std::greater<Event>> done;
  std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
  for (int i = 0; i < std::max(teams, 1); ++i) free_at.push(0.0);
  std::vector<uint32_t> next(U, 0), left(n_tasks);
  size_t total = 0;
  for (size_t i = 0; i < U; ++i) {
    total += n_tasks[i];
    if (n_deps[i] == 0) ready.push((int)i);
  }
  w.tasks.reserve(total);
  while (w.tasks.size() < total) {
    const double now = free_at.top();
    free_at.pop();
    while (!done.empty() && done.top().first <= now) {
      const int gid = done.top().second;
      done.pop();
      if (--left[gid] == 0)
        for (int s : succ[gid])
          if (--n_deps[s] == 0) ready.push(s);
    }
    if (ready.empty()) {
      if (done.empty()) fail(QTC_ERR_INVALID, "internal: units with unmet dependencies");
      free_at.push(done.top().first);   // idle until the next task ends
      continue;
    }
    const int gid = ready.top();
    GTask t = tmpl[gid];
    if (t.kind != GT_SMEM) t.b = next[gid];
    w.tasks.push_back(t);
    if (++next[gid] == n_tasks[gid]) ready.pop();
    done.push({now + dur[gid], gid});
    free_at.push(now + dur[gid]);
  }
  return w;
}

uint64_t runs_max(const GRuns& r, uint32_t bits) {
  // largest operand offset the run map produces over indices < 2^bits
  uint64_t off = 0;
  for (int k = 0; k < r.n; ++k)
    if (r.src[k] < bits) {
      const uint32_t len = std::min<uint32_t>(r.len[k], bits - r.src[k]);
      off |= (((uint64_t)1 << len) - 1) << r.dst[k];
    }
  return off;
}

uint64_t runs_offset_host(const GRuns& r, uint64_t idx) {
  uint64_t off = 0;
  for (int k = 0; k < r.n; ++k)
    off |= ((idx >> r.src[k]) & ((1ull << r.len[k]) - 1)) << r.dst[k];
  return off;
}

uint64_t positions_max(const uint8_t* pos, int n) {
  uint64_t off = 0;
  for (int i = 0; i < n; ++i)
    if (pos[i] != kAbsent) off |= (uint64_t)1 << pos[i];
  return off;
}

// Checks every access of a wave against its buffers and the task order
// against the dependencies, so that a lowering mistake is an error on the
// host instead of a bad address or a wait that never ends on the device.
void validate_wave(const WaveHost& w, uint32_t table_elems, uint32_t arena_elems,
                   size_t elem_of_wave, size_t work_bytes) {
  auto check_ref = [&](uint32_t off, bool global, uint64_t max_index, const char* what) {
    const uint64_t end = (uint64_t)off + max_index + 1;
    if (global) {
      if (end > w.global_elems) fail(QTC_ERR_INVALID, "internal: %s beyond the work buffer", what);
    } else if (off < table_elems) {
      if (end > table_elems) fail(QTC_ERR_INVALID, "internal: %s beyond the gate table", what);
    } else if (end > (uint64_t)table_elems + arena_elems) {
      fail(QTC_ERR_INVALID, "internal: %s beyond the task arena", what);
    }
  };
  for (const GTask& t : w.tasks) {
    if (t.wait_begin + t.wait_count > w.waits.size())
      fail(QTC_ERR_INVALID, "internal: wait list out of range");
    if (t.kind == GT_SMEM) {
      if ((uint64_t)t.a + t.b > w.ops.size()) fail(QTC_ERR_INVALID, "internal: op range");
      if (t.signal != 0xFFFFFFFFu && t.signal >= w.n_counters)
        fail(QTC_ERR_INVALID, "internal: signal counter out of range");
      for (uint32_t i = t.a; i < t.a + t.b; ++i) {
        const SOp& op = w.ops[i];
        if (op.code == SOP_CONTRACT) {
          uint64_t m1 = positions_max(op.p1, op.rc) | positions_max(op.y1, op.ry);
          uint64_t m2 = positions_max(op.p2, op.rc) | positions_max(op.y2, op.ry);
          check_ref(op.out, op.flags & SOPF_OUT_GLOBAL, ((uint64_t)1 << op.rc) - 1, "op output");
          check_ref(op.in1, op.flags & SOPF_IN1_GLOBAL, m1, "op operand 1");
          check_ref(op.in2, op.flags & SOPF_IN2_GLOBAL, m2, "op operand 2");
        } else if (op.code == SOP_LEAFGRAD) {
          check_ref(op.in1, false, ((uint64_t)1 << op.rc) - 1, "leaf adjoint");
          check_ref(op.in2, false, ((uint64_t)1 << op.rc) - 1, "leaf derivative");
        } else if (op.code == SOP_RESULT) {
          check_ref(op.in1, op.flags & SOPF_IN1_GLOBAL, 0, "result");
        } else if (op.code == SOP_SEED) {
          check_ref(op.out, op.flags & SOPF_OUT_GLOBAL, 0, "seed");
        }
      }
    } else if (t.kind == GT_TC) {
      if (t.a >= w.tsteps.size()) fail(QTC_ERR_INVALID, "internal: GEMM index");
      const TStep& ts = w.tsteps[t.a];
      if (t.b >= (((uint64_t)ts.m_tiles * ts.n_tiles) << ts.bb))
        fail(QTC_ERR_INVALID, "internal: GEMM tile index");
    } else {
      if (t.a >= w.steps.size()) fail(QTC_ERR_INVALID, "internal: step index");
      const GStep& st = w.steps[t.a];
      if (t.b >= st.n_chunks) fail(QTC_ERR_INVALID, "internal: chunk index");
    }
  }
  for (const TStep& ts : w.tsteps) {
    check_ref(ts.a_off, true, runs_max(ts.am, ts.mb) | runs_max(ts.ak, ts.kb) |
                                  runs_max(ts.ab, ts.bb), "GEMM operand A");
    check_ref(ts.b_off, true, runs_max(ts.bk, ts.kb) | runs_max(ts.bn, ts.nb) |
                                  runs_max(ts.bbt, ts.bb), "GEMM operand B");
    check_ref(ts.c_off, true, runs_max(ts.cm, ts.mb) | runs_max(ts.cn, ts.nb) |
                                  runs_max(ts.cb, ts.bb), "GEMM output");
    if (ts.done_ctr >= w.n_counters) fail(QTC_ERR_INVALID, "internal: GEMM counter");
    if (ts.nb < 6 || ((1ull << ts.nb) % kTcCols)) fail(QTC_ERR_INVALID, "internal: GEMM N");
  }
  for (const GStep& st : w.steps) {
    if (st.flags & GSF_TILE) {
      const GTileMap& t = st.tile;
      const bool sa = (t.staged & 1) != 0, sb = (t.staged & 2) != 0;
      const bool ga = !(st.flags & GSF_A_TABLE), gbl = !(st.flags & GSF_B_TABLE);
      if ((sa && !ga) || (sb && !gbl)) fail(QTC_ERR_INVALID, "internal: a table operand staged");
      if (t.nv != 8 + t.kout + t.ns || t.kout > kTileMaxOut || t.ns > kTileMaxRegSum)
        fail(QTC_ERR_INVALID, "internal: tile bit split");
      const uint64_t ta = runs_max(t.tfa, t.nv), tb = runs_max(t.tfb, t.nv);
      const uint64_t tc = runs_max(t.tfc, t.nv);
      if (sa && ta >= (1ull << t.nfa)) fail(QTC_ERR_INVALID, "internal: tile beyond footprint A");
      if (sb && tb >= (1ull << t.nfb)) fail(QTC_ERR_INVALID, "internal: tile beyond footprint B");
      if (tc >= (1ull << t.nfc)) fail(QTC_ERR_INVALID, "internal: tile beyond footprint C");
      const uint64_t ea = runs_max(t.oa, t.no) | runs_max(t.qa, t.nq) |
                          (sa ? runs_max(t.ffa, t.nfa) : ta);
      const uint64_t eb = runs_max(t.ob, t.no) | runs_max(t.qb, t.nq) |
                          (sb ? runs_max(t.ffb, t.nfb) : tb);
      check_ref(st.a_off, ga, ea, "tile operand A");
      check_ref(st.b_off, gbl, eb, "tile operand B");
      if (!(st.flags & GSF_LEAFGRAD))
        check_ref(st.c_off, true, runs_max(t.oc, t.no) | runs_max(t.ffc, t.nfc), "tile output");
      else
        check_ref(st.der_off, false, runs_max(t.ffc, t.nfc), "leaf derivative");
      if (!(st.flags & GSF_SPLIT)) {
        const uint64_t no = 1ull << t.no;
        if (t.o_per_chunk == 0 || (uint64_t)st.n_chunks * t.o_per_chunk < no ||
            (uint64_t)(st.n_chunks - 1) * t.o_per_chunk >= no || t.q_per_chunk != (1ull << t.nq))
          fail(QTC_ERR_INVALID, "internal: tile chunks do not cover the outputs");
      }
      if (st.flags & GSF_SPLIT) {
        if (t.no != 0) fail(QTC_ERR_INVALID, "internal: split tile with outer outputs");
        if (t.q_per_chunk == 0 || (uint64_t)st.n_chunks * t.q_per_chunk < (1ull << t.nq))
          fail(QTC_ERR_INVALID, "internal: tile chunks do not cover the summed values");
        check_ref(st.partial_off, true, ((uint64_t)st.n_chunks << t.nfc) - 1, "tile partials");
        if (st.arrive_ctr >= w.n_counters) fail(QTC_ERR_INVALID, "internal: arrive counter");
      }
      if (tile_region_bytes(st, elem_of_wave) > work_bytes)
        fail(QTC_ERR_INVALID, "internal: tile footprints beyond the team's shared memory");
      if (st.done_ctr >= w.n_counters) fail(QTC_ERR_INVALID, "internal: done counter");
      continue;
    }
    if (st.flags & (GSF_YPAIR | GSF_LANES_Y)) {
      auto low_run = [](const GRuns& r) {
        return (r.n > 0 && r.src[0] == 0 && r.dst[0] == 0) ? (int)r.len[0] : 0;
      };
      if (st.flags & (GSF_A_TABLE | GSF_B_TABLE))
        fail(QTC_ERR_INVALID, "internal: paired or lane-summed step on a table operand");
      if ((st.flags & GSF_YPAIR) &&
          (low_run(st.ya) < 1 || low_run(st.yb) < 1 || (st.a_off & 1u) || (st.b_off & 1u) ||
           ((st.flags & GSF_SPLIT) && (!(st.flags & GSF_LANES_Y) || (st.chunk & 1u)))))
        fail(QTC_ERR_INVALID, "internal: paired loads without adjacent summed pairs");
      if ((st.flags & GSF_LANES_Y) && !(st.flags & GSF_SPLIT))
        fail(QTC_ERR_INVALID, "internal: lanes over the summed index outside a split step");
    }
    if (st.flags & GSF_ROWS) {
      // rows in groups along output bits that one operand lacks; the row
      // order a bijection of the row bits
      const int row0 = 8, nrb = (int)st.rc - row0;
      const uint64_t ny = 1ull << st.ry;
      const bool fixed = st.share == GRS_FIXA || st.share == GRS_FIXB;
      const int g = fixed ? grs_fix_bits((uint32_t)ny) : 2;
      const uint32_t grp = 1u << g;
      bool ok = nrb >= g && kGRow == (1u << row0) &&
                !(st.flags & (GSF_SPLIT | GSF_TILE | GSF_LEAFGRAD)) &&
                !(fixed && (st.flags & GSF_YPAIR)) &&
                (fixed ? ny <= 4 : (ny >= 8 && ny <= kYTab && st.share >= GRS_ZX &&
                                    st.share <= GRS_XX &&
                                    !(st.flags & (GSF_A_TABLE | GSF_B_TABLE)))) &&
                st.chunk >= grp && st.chunk % grp == 0 &&
                (uint64_t)st.n_chunks * st.chunk == (1ull << nrb);
      uint64_t seen = 0;
      for (int i = 0; ok && i < nrb; ++i) {
        const uint64_t o = runs_offset_host(st.rows, 1ull << i);
        ok = o != 0 && (o & (o - 1)) == 0 && o < (1ull << nrb) && !(seen & o);
        seen |= o;
      }
      // counter bit i of a group: missing from A (zm) or from B (xm)
      const int zm = st.share == GRS_ZX ? 1 : st.share == GRS_ZZ ? 3
                     : st.share == GRS_FIXA ? (int)grp - 1 : 0;
      const int xm = st.share == GRS_ZX ? 2 : st.share == GRS_XX ? 3
                     : st.share == GRS_FIXB ? (int)grp - 1 : 0;
      for (int i = 0; ok && i < g; ++i) {
        const uint64_t bit = runs_offset_host(st.rows, 1ull << i) << row0;
        if ((zm >> i) & 1) ok = runs_offset_host(st.ca, bit) == 0;
        if (ok && ((xm >> i) & 1)) ok = runs_offset_host(st.cb, bit) == 0;
      }
      if (!ok) fail(QTC_ERR_INVALID, "internal: shared rows on an unfit step");
    }
    const uint64_t ma = runs_max(st.ca, st.rc) | runs_max(st.ya, st.ry);
    const uint64_t mb = runs_max(st.cb, st.rc) | runs_max(st.yb, st.ry);
    check_ref(st.a_off, !(st.flags & GSF_A_TABLE), ma, "step operand A");
    check_ref(st.b_off, !(st.flags & GSF_B_TABLE), mb, "step operand B");
    if (!(st.flags & GSF_LEAFGRAD))
      check_ref(st.c_off, true, ((uint64_t)1 << st.rc) - 1, "step output");
    else
      check_ref(st.der_off, false, ((uint64_t)1 << st.rc) - 1, "leaf derivative");
    if (st.flags & GSF_SPLIT) {
      if (st.rc > 8) fail(QTC_ERR_INVALID, "internal: split step with more than 256 outputs");
      check_ref(st.partial_off, true, ((uint64_t)st.n_chunks << st.rc) - 1, "partials");
      if (st.arrive_ctr >= w.n_counters) fail(QTC_ERR_INVALID, "internal: arrive counter");
      if (st.chunk > kYTab) fail(QTC_ERR_INVALID, "internal: split chunk above the table");
    } else if (st.chunk > kMaxChunkRows) {
      fail(QTC_ERR_INVALID, "internal: chunk of more rows than the row table");
    } else if (((uint64_t)st.chunk * std::min<uint64_t>((uint64_t)1 << st.rc, kGRow)) == 0) {
      fail(QTC_ERR_INVALID, "internal: empty chunk");
    }
    if (st.done_ctr >= w.n_counters) fail(QTC_ERR_INVALID, "internal: done counter");
  }
  // every wait refers to a counter whose producer tasks all come earlier
  std::vector<int64_t> last_producer(w.n_counters, -1);
  for (size_t i = 0; i < w.tasks.size(); ++i) {
    const GTask& t = w.tasks[i];
    for (uint32_t k = 0; k < t.wait_count; ++k) {
      const WaitDev& wd = w.waits[t.wait_begin + k];
      if (wd.counter >= w.n_counters) fail(QTC_ERR_INVALID, "internal: wait counter");
      if (last_producer[wd.counter] < 0)
        fail(QTC_ERR_INVALID, "internal: task %zu waits for a producer that comes later", i);
    }
    if (t.kind == GT_SMEM) {
      if (t.signal != 0xFFFFFFFFu) last_producer[t.signal] = (int64_t)i;
    } else if (t.kind == GT_TC) {
      const TStep& ts = w.tsteps[t.a];
      if (t.b + 1 == (((uint64_t)ts.m_tiles * ts.n_tiles) << ts.bb))
        last_producer[ts.done_ctr] = (int64_t)i;
    } else {
      const GStep& st = w.steps[t.a];
      // a step is complete only after its last chunk; mark it at the last chunk
      if (t.b + 1 == st.n_chunks) last_producer[st.done_ctr] = (int64_t)i;
    }
  }
}

}  // namespace

void build_graph_program(HostProgram& hp, const std::vector<Plan>& plans,
                         const std::vector<std::vector<int>>& leaf_gate,
                         const std::vector<uint32_t>& val_off,
                         const std::vector<uint32_t>& der_off, size_t max_dynamic,
                         const ProgramOptions& opts) {
  const size_t elem = elem_bytes(hp.dtype);
  const size_t wave_cap_bytes = opts.wave_cap_bytes;
  const int N = (int)plans.size();
  GraphLimits lim;
  lim.arena_elems = (uint32_t)(49152 / elem);
  lim.subtree_elems = (uint64_t)opts.subtree_bytes / elem;
  lim.task_terms_log2 = opts.task_terms_log2;
  lim.tile_mode = opts.tile_mode;
  lim.elem = elem;
  if (opts.small_rank > 0) lim.small_rank = opts.small_rank;
  lim.tensor_cores = hp.dtype == QTC_SPLIT_BF16;
  if (lim.tensor_cores) lim.tile_mode = 0;   // the tensor-core build has no tile tasks
  // with tensor cores four teams share one CTA's shared memory
  if (lim.tensor_cores) lim.arena_elems = (uint32_t)(32768 / elem);
  std::vector<NetGraph> graphs(N);
  for (int i = 0; i < N; ++i) {
    // a network that fits whole in shared memory stays one fused task
    LoweredNet ln = lower_smem(plans[i], leaf_gate[i], val_off, der_off, hp.table_elems,
                               hp.want_grad != 0, hp.table_elems + lim.arena_elems);
    if (ln.fits && !opts.force_graph) {
      GUnit u;
      u.kind = GT_SMEM;
      u.ops = std::move(ln.ops);
      u.arena_elems = ln.arena_elems;
      graphs[i].units.push_back(std::move(u));
      continue;
    }
    // a subtree that does not fit its arena is cut into smaller ones
    GraphLimits li = lim;
    for (;;) {
      graphs[i] = lower_graph(plans[i], leaf_gate[i], val_off, der_off, hp.table_elems,
                              hp.want_grad != 0, li);
      if (graphs[i].fits || li.subtree_elems <= 64) break;
      li.subtree_elems /= 2;
    }
    if (!graphs[i].fits)
      fail(QTC_ERR_UNSUPPORTED, "network %d (max rank %d): %s", i, plans[i].max_rank,
           graphs[i].why.c_str());
    // a network whose stored values exceed the wave limit on their own:
    // checkpoint segments, recomputed by the adjoint sweep (fewest that fit)
    const uint64_t cap_elems = wave_cap_bytes / elem;
    auto over = [&](const NetGraph& g) {
      return ((g.global_elems + 63) & ~uint64_t(63)) > cap_elems;
    };
    if (over(graphs[i])) {
      // reuse memory also where that adds write-after-read dependencies
      GraphLimits ld = li;
      ld.reuse_with_deps = true;
      NetGraph g = lower_graph(plans[i], leaf_gate[i], val_off, der_off, hp.table_elems,
                               hp.want_grad != 0, ld);
      if (g.fits && g.global_elems < graphs[i].global_elems) {
        graphs[i] = std::move(g);
        li = ld;
      }
    }
    if (hp.want_grad && over(graphs[i])) {
      for (int k : {2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64}) {
        GraphLimits lk = li;
        lk.reuse_with_deps = true;
        lk.checkpoint_segments = k;
        NetGraph g = lower_graph(plans[i], leaf_gate[i], val_off, der_off, hp.table_elems,
                                 true, lk);
        if (!g.fits) break;
        const bool ok = ((g.global_elems + 63) & ~uint64_t(63)) <= cap_elems;
        if (ok || g.global_elems < graphs[i].global_elems) graphs[i] = std::move(g);
        if (ok) break;
      }
    }
    check_global_placement(graphs[i]);
    hp.max_checkpoint_segments = std::max(hp.max_checkpoint_segments,
                                          graphs[i].checkpoint_segments);
    hp.sum_global_elems += graphs[i].global_elems;
    hp.sum_unshared_elems += graphs[i].unshared_elems;
  }
  // waves: largest networks first, first fit under the cap
  const uint64_t cap = wave_cap_bytes / elem;
  std::vector<int> order(N);
  for (int i = 0; i < N; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return graphs[a].global_elems > graphs[b].global_elems;
  });
  std::vector<std::vector<int>> waves;
  std::vector<uint64_t> used;
  for (int i : order) {
    const uint64_t need = (graphs[i].global_elems + 63) & ~uint64_t(63);
    if (need > cap)
      fail(QTC_ERR_ARENA,
           "network %d needs %llu bytes of intermediates in global memory, more than the wave "
           "limit of %zu bytes",
           i, (unsigned long long)(need * elem), wave_cap_bytes);
    size_t w = 0;
    while (w < waves.size() && used[w] + need > cap) ++w;
    if (w == waves.size()) {
      waves.emplace_back();
      used.push_back(0);
    }
    waves[w].push_back(i);
    used[w] += need;
  }
  hp.graph = true;
  hp.waves.clear();
  uint32_t max_arena = 0;
  for (const NetGraph& g : graphs)
    for (const GUnit& u : g.units) max_arena = std::max(max_arena, u.arena_elems);
  hp.tensor_cores = false;
  for (auto& wnets : waves) {
    std::sort(wnets.begin(), wnets.end());
    hp.waves.push_back(assemble_wave(wnets, graphs, elem, opts.sm_count * 4));

    if (!hp.waves.back().tsteps.empty()) hp.tensor_cores = true;
    hp.max_global_elems = std::max(hp.max_global_elems, hp.waves.back().global_elems);
    hp.max_counters = std::max(hp.max_counters, hp.waves.back().n_counters);
  }
  hp.max_arena = max_arena;
  hp.stage_ops = 32;
  auto round16 = [](size_t x) { return (uint32_t)((x + 15) & ~size_t(15)); };
  const size_t smem_task = (size_t)hp.stage_ops * sizeof(SOp) + (size_t)max_arena * elem;
  const size_t chunk_task = 2 * (size_t)kYTab * sizeof(uint32_t) + 256 * elem +
                            3 * (size_t)kMaxChunkRows * sizeof(uint32_t);
  size_t tile_task = 0;
  hp.tiles = false;
  for (const WaveHost& w : hp.waves)
    for (const GStep& st : w.steps)
      if (st.flags & GSF_TILE) {
        tile_task = std::max(tile_task, tile_region_bytes(st, elem));
        hp.tiles = true;
      }
  hp.work_bytes = round16(std::max({smem_task, chunk_task, tile_task}));
  hp.table_bytes = round16((size_t)hp.table_elems * elem);
  hp.smem = hp.table_bytes + (size_t)(hp.tensor_cores ? 4 : 1) * hp.work_bytes;
  for (const WaveHost& w : hp.waves) validate_wave(w, hp.table_elems, max_arena, elem, hp.work_bytes);
  if (hp.smem > max_dynamic)
    fail(QTC_ERR_UNSUPPORTED, "graph program needs %zu bytes of shared memory (limit %zu)",
         hp.smem, max_dynamic);
}

}  // namespace qtc
