// Gate fusion (Sec. III.B).
//
// The paper's fuser works in two steps: small gates are absorbed into large
// neighbours on the same qubits, then gates close in space and time are
// greedily grown up to the maximum fuse size f.  This fuser reaches the same
// kind of result with one rule applied greedily in time order: a later
// fused gate b may be pulled back into fused gate a when
//   (1) no fused gate between a and b (that stays in place) touches b's
//       qubits, so b commutes to a's position, and
//   (2) the union of their qubits has at most f qubits.
// Phase 1 only grows a by gates that share at least one qubit with it (the
// paper's "nearest neighbours"); phase 2 then packs gates that are disjoint,
// which still saves a full pass over the state per merge.  Channels are
// fused like gates of their qubits ("slots"): the operator in a slot is
// chosen per trajectory.  Which candidate a grows by is a choice the paper
// leaves open: two rules are run (most shared qubits; most later gates
// absorbed), each on the circuit and on its time reversal, and the plan
// with the lower modelled pass time is kept.
#include <algorithm>
#include <bit>
#include <new>

#include "qt_internal.h"

namespace qt {

namespace {

struct Work {
  uint64_t mask;
  std::vector<uint32_t> members;
  bool alive;
};

int popc(uint64_t x) { return std::popcount(x); }

// Grow gate a by pulling later gates back into it.  allow_disjoint: also
// accept gates sharing no qubit with a.
enum class Pick { kShared, kLookahead };

// Grow gate a by pulling later gates back into it.  allow_disjoint: also
// accept gates sharing no qubit with a.  Among the gates that may join, a
// gate on a subset of a's qubits is taken at once; otherwise the rule picks
// the candidate sharing the most qubits with a (kShared), or the one after
// which the most later gates would fall inside the merged qubit set
// (kLookahead, within a window of 256 gates), earliest first on ties.
bool grow(std::vector<Work>& g, size_t a, int kmax, uint64_t all_mask, bool allow_disjoint, Pick pick) {
  bool changed = false;
  for (;;) {
    uint64_t blocked = 0;
    long cand = -1;
    int cand_score = 0;
    for (size_t b = a + 1; b < g.size(); ++b) {
      if (!g[b].alive) continue;
      const uint64_t qb = g[b].mask;
      if ((qb & blocked) == 0) {
        const uint64_t un = g[a].mask | qb;
        // an op wider than the fuse size forms its own gate; it still absorbs
        // gates on a subset of its qubits
        if (popc(un) <= std::max(kmax, popc(g[a].mask))) {
          if ((qb & ~g[a].mask) == 0) {      // no growth: take it now
            g[a].members.insert(g[a].members.end(), g[b].members.begin(), g[b].members.end());
            g[b].alive = false;
            changed = true;
            continue;
          }
          if (allow_disjoint || (qb & g[a].mask) != 0) {
            int score = popc(qb & g[a].mask);
            if (pick == Pick::kLookahead) {
              uint64_t blk = 0;
              int absorbed = 0, seen = 0;
              for (size_t c = a + 1; c < g.size() && seen < 256; ++c) {
                if (!g[c].alive || c == b) continue;
                ++seen;
                const uint64_t qc = g[c].mask;
                if ((qc & blk) == 0 && (qc & ~un) == 0) ++absorbed;
                else blk |= qc;
              }
              score += 64 * absorbed;
            }
            if (cand < 0 || score > cand_score) { cand = static_cast<long>(b); cand_score = score; }
          }
        }
      }
      blocked |= qb;
      if (blocked == all_mask) break;      // every later gate is blocked
    }
    if (cand < 0) return changed;
    Work& wb = g[static_cast<size_t>(cand)];
    g[a].members.insert(g[a].members.end(), wb.members.begin(), wb.members.end());
    g[a].mask |= wb.mask;
    wb.alive = false;
    changed = true;
  }
}

// relative device time of one pass of a fused gate of width w (measured
// rates of the fused-gate kernels at 30 qubits: 6.5 TB/s up to width 3,
// 5.9 at width 4, and 4.5 and 3.9 for the tensor-core kernel at widths 5, 6)
double pass_cost(int w) {
  static const double c[7] = {1.0, 1.0, 1.0, 1.0, 1.1, 1.45, 1.7};
  return c[w < 7 ? w : 6];
}

}  // namespace

qt_status fuse_circuit(const Circuit& c, uint32_t kmax, Fused& f) {
  f.c = &c;
  f.kmax = kmax;
  f.gates.clear();
  f.gate_ops = 0;
  std::vector<Work> g;
  g.reserve(c.ops.size());
  for (uint32_t i = 0; i < c.ops.size(); ++i) {
    const Op& op = c.ops[i];
    uint64_t m = 0;
    for (uint32_t b = 0; b < op.q; ++b) m |= 1ull << op.qubits[b];
    g.push_back(Work{m, {i}, true});
    if (op.kind == QT_OP_GATE) f.gate_ops++;
  }
  const uint64_t all_mask = (c.n >= 64) ? ~0ull : ((1ull << c.n) - 1ull);
  // four plans: each candidate rule on the circuit and on its time reversal;
  // keep the one with the lower pass cost.  A plan of the reversed circuit,
  // taken in reverse order with each gate's members in circuit order, is a
  // plan of the circuit: every reordering it implies swaps operations on
  // disjoint qubits.
  std::vector<Work> best;
  double best_cost = 0.0;
  for (int reversed = 0; reversed < 2; ++reversed)
    for (Pick pick : {Pick::kShared, Pick::kLookahead}) {
      std::vector<Work> w = g;
      if (reversed) std::reverse(w.begin(), w.end());
      for (int phase = 0; phase < 2; ++phase)
        for (size_t a = 0; a < w.size(); ++a)
          if (w[a].alive) grow(w, a, static_cast<int>(kmax), all_mask, phase == 1, pick);
      double cost = 0.0;
      for (const Work& x : w)
        if (x.alive) cost += pass_cost(popc(x.mask));
      if (best.empty() || cost < best_cost - 1e-9) {
        if (reversed) {
          std::reverse(w.begin(), w.end());
          for (Work& x : w) std::sort(x.members.begin(), x.members.end());
        }
        best = std::move(w);
        best_cost = cost;
      }
    }
  g = std::move(best);

  f.gate_of_op.assign(c.ops.size(), 0);
  for (const Work& w : g) {
    if (!w.alive) continue;
    FusedGate fg;
    for (uint32_t q = 0; q < 64; ++q)
      if (w.mask & (1ull << q)) fg.targets.push_back(q);
    fg.members = w.members;
    std::vector<std::pair<uint32_t, const cd*>> seq;
    for (uint32_t m : fg.members) {
      const Op& op = c.ops[m];
      if (op.kind != QT_OP_GATE) fg.has_channel = true;
      seq.emplace_back(m, op.mat(op.kind == QT_OP_GATE ? 0 : static_cast<uint32_t>(op.def)));
      f.gate_of_op[m] = static_cast<uint32_t>(f.gates.size());
    }
    compose(c, fg.targets, seq, fg.def);
    f.gates.push_back(std::move(fg));
  }
  return QT_OK;
}

}  // namespace qt

using namespace qt;

extern "C" {

qt_status qt_fuse(const qt_circuit* c, uint32_t max_fused_qubits, qt_fused** out) {
  clear_error();
  if (!c || !out) return set_error(QT_ERR_INVALID_ARG, "qt_fuse: NULL argument");
  *out = nullptr;
  uint32_t k = max_fused_qubits;
  if (k == 0) k = c->n >= 20 ? 4 : (c->n >= 12 ? 3 : 2);   // automatic: f=4 for large states
  if (k > QT_MAX_FUSED_QUBITS) return set_error(QT_ERR_INVALID_ARG, "qt_fuse: max_fused_qubits %u > 6", k);
  k = std::min<uint32_t>(k, c->n);
  qt_fused* f = new (std::nothrow) qt_fused();
  if (!f) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_fuse: host allocation");
  const qt_status s = fuse_circuit(*c, k, *f);
  if (s != QT_OK) {
    delete f;
    return s;
  }
  *out = f;
  return QT_OK;
}

void qt_fused_destroy(qt_fused* f) { delete f; }

qt_status qt_fused_info(const qt_fused* f, qt_fused_info_t* out) {
  clear_error();
  if (!f || !out) return set_error(QT_ERR_INVALID_ARG, "qt_fused_info: NULL argument");
  out->num_fused = static_cast<uint32_t>(f->gates.size());
  out->max_width = 0;
  for (const auto& g : f->gates) out->max_width = std::max<uint32_t>(out->max_width, g.targets.size());
  out->num_ops = static_cast<uint32_t>(f->c->ops.size());
  out->num_channels = static_cast<uint32_t>(f->c->channel_op.size());
  return QT_OK;
}

qt_status qt_fused_gate(const qt_fused* f, uint32_t g, uint32_t* width, uint32_t* targets,
                        uint32_t* num_members, uint32_t* members, size_t cap, double* matrix) {
  clear_error();
  if (!f) return set_error(QT_ERR_INVALID_ARG, "qt_fused_gate: NULL fused");
  if (g >= f->gates.size()) return set_error(QT_ERR_INVALID_ARG, "qt_fused_gate: index %u out of range", g);
  const FusedGate& fg = f->gates[g];
  if (width) *width = static_cast<uint32_t>(fg.targets.size());
  if (targets)
    for (size_t i = 0; i < fg.targets.size(); ++i) targets[i] = fg.targets[i];
  if (num_members) *num_members = static_cast<uint32_t>(fg.members.size());
  if (members)
    for (size_t i = 0; i < fg.members.size() && i < cap; ++i) members[i] = fg.members[i];
  if (matrix)
    for (size_t e = 0; e < fg.def.size(); ++e) {
      matrix[2 * e] = fg.def[e].real();
      matrix[2 * e + 1] = fg.def[e].imag();
    }
  return QT_OK;
}

}  // extern "C"
