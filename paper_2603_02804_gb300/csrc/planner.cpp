// Fusion planner: turns a gate list into passes over shared-memory tiles.
//
// Forward fusion (Sec. 3.2) is generalised from "consecutive gates on the
// same or adjacent qubits" to "every gate whose dependencies are met and whose
// qubit lies in the current 4-qubit register group", with diagonal gates
// (RZ, CZ) allowed to commute past each other. The backward program is the
// exact reverse of the forward one, with each fused 2x2 expanded back into
// its rotations so every parameter gets its own gradient term (Sec. 3.3).
#include "planner.h"

#include <limits>

#include <algorithm>
#include <cstdlib>
#include <functional>
#include <set>
#include <stdexcept>
#include <string>

namespace qf {

namespace {

bool is_diag(int kind) { return kind == G_RZ || kind == G_CZ; }
bool is_rot(int kind) { return kind == G_RX || kind == G_RY || kind == G_RZ; }

struct Dag {
  std::vector<int> indeg;
  std::vector<std::vector<int>> succ;
};

// Gate b depends on an earlier gate a when they share a qubit and are not
// both diagonal (diagonal gates commute with each other).
Dag build_dag(const Circuit& c) {
  const int M = (int)c.gates.size();
  Dag d;
  d.indeg.assign(M, 0);
  d.succ.assign(M, {});
  std::vector<int> last_nd(c.n, -1);
  std::vector<std::vector<int>> diag_since(c.n);
  for (int g = 0; g < M; ++g) {
    const Gate& gt = c.gates[g];
    int qs[2] = {gt.q0, (gt.kind == G_CZ || gt.kind == G_CNOT) ? gt.q1 : -1};
    std::vector<int> deps;
    for (int q : qs) {
      if (q < 0) continue;
      if (last_nd[q] >= 0) deps.push_back(last_nd[q]);
      if (!is_diag(gt.kind)) deps.insert(deps.end(), diag_since[q].begin(), diag_since[q].end());
    }
    for (int q : qs) {
      if (q < 0) continue;
      if (is_diag(gt.kind)) {
        diag_since[q].push_back(g);
      } else {
        last_nd[q] = g;
        diag_since[q].clear();
      }
    }
    std::sort(deps.begin(), deps.end());
    deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
    for (int a : deps) {
      d.succ[a].push_back(g);
      d.indeg[g]++;
    }
  }
  return d;
}

// Absorption state with an undo log so candidate passes can be tried.
struct Sim {
  const Circuit* c;
  const Dag* dag;
  std::vector<int> indeg;
  std::vector<char> done;
  std::set<int> front;  // ready, not yet absorbed
  std::vector<int> log;
  int n_done = 0;

  Sim(const Circuit& cc, const Dag& d) : c(&cc), dag(&d), indeg(d.indeg), done(d.indeg.size(), 0) {
    for (int g = 0; g < (int)indeg.size(); ++g)
      if (indeg[g] == 0) front.insert(g);
  }
  void absorb(int g) {
    done[g] = 1;
    ++n_done;
    front.erase(g);
    log.push_back(g);
    for (int s : dag->succ[g])
      if (--indeg[s] == 0) front.insert(s);
  }
  void undo_to(size_t mark) {
    while (log.size() > mark) {
      int g = log.back();
      log.pop_back();
      for (int s : dag->succ[g])
        if (indeg[s]++ == 0) front.erase(s);
      done[g] = 0;
      --n_done;
      front.insert(g);
    }
  }
};

// Absorb, round by round, every ready gate that is a CZ or a rotation on a
// qubit of `group`. At most `max_slots` rotations. Returns a score that
// weighs rotations (the real work) above sign-only CZs.
int absorb_step(Sim& s, uint64_t group, int max_slots, std::vector<int>* out) {
  int rot = 0, cz = 0;
  bool progress = true;
  std::vector<int> cand;
  while (progress) {
    progress = false;
    cand.assign(s.front.begin(), s.front.end());
    for (int g : cand) {
      if (s.done[g] || s.indeg[g] != 0) continue;
      const Gate& gt = s.c->gates[g];
      if (gt.kind == G_CZ) {
        ++cz;
      } else if (gt.kind == G_CNOT) {
        // a permutation of the target's register pairs; the control may be any qubit
        if (!((group >> gt.q1) & 1)) continue;
        ++cz;
      } else {
        if (!((group >> gt.q0) & 1)) continue;
        if (rot >= max_slots) continue;
        ++rot;
      }
      s.absorb(g);
      if (out) out->push_back(g);
      progress = true;
    }
  }
  return rot * 64 + cz;
}

// One item of a round: the next run of rotations on one qubit, either a run
// of diagonal rotations ("pre", when the qubit's next rotation is an RZ) or
// one RY followed by the diagonal rotations that become ready after it.
struct ItemRec {
  std::vector<int> pre;
  int y = -1;
  std::vector<int> post;
  bool empty() const { return pre.empty() && y < 0; }
};

struct RoundRec {
  ItemRec it[4];
  std::vector<int> czs;
};

struct StepRec {
  int group;
  std::vector<int> gates;        // every gate absorbed by the step
  std::vector<RoundRec> rounds;  // round programs only
};

struct Tile {
  std::vector<int> local_to_global;  // size K
  std::vector<std::vector<int>> groups;  // local bits per group (4 each)
  std::vector<uint64_t> group_qmask;     // global qubit masks
};

Tile make_tile(const std::vector<int>& globals_sorted, int K) {
  Tile t;
  t.local_to_global = globals_sorted;
  // groups: local nibbles; the last one top-aligned when K is not a multiple of 4
  for (int base = 0; base < K; base += 4) {
    int b = base + 4 <= K ? base : K - 4;
    std::vector<int> g = {b, b + 1, b + 2, b + 3};
    t.groups.push_back(g);
  }
  for (auto& g : t.groups) {
    uint64_t m = 0;
    for (int lb : g) m |= 1ull << t.local_to_global[lb];
    t.group_qmask.push_back(m);
  }
  return t;
}

int run_pass(Sim& s, const Tile& t, std::vector<StepRec>* steps) {
  int total = 0;
  for (;;) {
    int best = -1, best_score = 0;
    for (int gi = 0; gi < (int)t.groups.size(); ++gi) {
      size_t mark = s.log.size();
      int sc = absorb_step(s, t.group_qmask[gi], kMaxStepSlots, nullptr);
      s.undo_to(mark);
      if (sc > best_score) {
        best_score = sc;
        best = gi;
      }
    }
    if (best < 0) break;
    std::vector<int> gs;
    total += absorb_step(s, t.group_qmask[best], kMaxStepSlots, steps ? &gs : nullptr);
    if (steps) steps->push_back({best, std::move(gs), {}});
  }
  return total;
}

// ---- round programs -------------------------------------------------------------
// Rotations of every qubit in circuit order, with a cursor that only lags the
// committed absorption state (simulated absorption may run ahead of it).
struct QubitRots {
  std::vector<std::vector<int>> rots;
  std::vector<size_t> cursor;
  int next(const Sim& s, int q) const {
    const auto& l = rots[q];
    size_t i = cursor[q];
    while (i < l.size() && s.done[l[i]]) ++i;
    return i < l.size() ? l[i] : -1;
  }
  // rotations of qubit q absorbed so far (its progress)
  int pos(const Sim& s, int q) const {
    const auto& l = rots[q];
    size_t i = cursor[q];
    while (i < l.size() && s.done[l[i]]) ++i;
    return (int)i;
  }
  void commit(const Sim& s) {
    for (size_t q = 0; q < rots.size(); ++q)
      while (cursor[q] < rots[q].size() && s.done[rots[q][cursor[q]]]) ++cursor[q];
  }
};

// The same tile with its free qubits (local bits 4..K-1) grouped by progress:
// sorted by their next pending rotation, then cut into groups of 4, each
// sorted ascending so that chain neighbours inside a group sit on adjacent
// register bits (the round programs apply register-register CZs between
// adjacent register bits only). Local bits 0..3 stay global qubits 0..3.
// Qubits at the same depth of the frontier then share a group, so round
// steps on them stay full where a staircase frontier crosses the nibbles.
Tile make_tile_by_progress(const std::vector<int>& globals_sorted, int K, const Sim& s, const QubitRots& qr) {
  std::vector<std::pair<long, int>> fr;
  for (int i = 4; i < K; ++i) {
    const int q = globals_sorted[i];
    const int g = qr.next(s, q);
    fr.push_back({g < 0 ? (1l << 40) : (long)g, q});
  }
  std::stable_sort(fr.begin(), fr.end());
  std::vector<int> order(globals_sorted.begin(), globals_sorted.begin() + 4);
  for (size_t c = 0; c < fr.size(); c += 4) {
    std::vector<int> grp;
    for (size_t k = c; k < std::min(fr.size(), c + 4); ++k) grp.push_back(fr[k].second);
    std::sort(grp.begin(), grp.end());
    order.insert(order.end(), grp.begin(), grp.end());
  }
  return make_tile(order, K);
}

bool ready(const Sim& s, int g) { return g >= 0 && !s.done[g] && s.indeg[g] == 0; }

// Absorb the next item of qubit q; false if its next rotation is not ready.
bool take_item(Sim& s, const QubitRots& qr, int q, ItemRec* it) {
  int g = qr.next(s, q);
  if (!ready(s, g)) return false;
  const auto& gates = s.c->gates;
  if (gates[g].kind == G_RZ) {
    while (ready(s, g) && gates[g].kind == G_RZ) {
      s.absorb(g);
      it->pre.push_back(g);
      g = qr.next(s, q);
    }
    return true;
  }
  s.absorb(g);
  it->y = g;
  g = qr.next(s, q);
  while (ready(s, g) && gates[g].kind == G_RZ) {
    s.absorb(g);
    it->post.push_back(g);
    g = qr.next(s, q);
  }
  return true;
}

bool has_rotations_left(const Sim& s, const QubitRots& qr, int q) { return qr.next(s, q) >= 0; }

// One round on the group's qubits. full: every qubit of the group that still
// has rotations must contribute an item, except a qubit shared with an
// earlier, overlapping group (not in `home`) that is already ahead of the
// group's own qubits (its next rotation comes later in the circuit than
// theirs). cap_pos >= 0 (a catch-up round, partial): only qubits with at
// most cap_pos rotations done contribute, so that lagging qubits catch up and
// full rounds resume. Ready CZs are absorbed at its end.
bool form_round(Sim& s, const QubitRots& qr, const int (&qs)[4], bool full, RoundRec* rr, int* n_rot,
                uint32_t home = 0xFu, int cap_pos = -1) {
  const size_t mark = s.log.size();
  long home_next = -1;
  for (int k = 0; k < 4; ++k)
    if ((home >> k) & 1u) home_next = std::max(home_next, (long)qr.next(s, qs[k]));
  RoundRec r;
  int items = 0, want = 0, got = 0, rot = 0;
  for (int k = 0; k < 4; ++k) {
    bool dup = false;
    for (int j = 0; j < k; ++j) dup |= qs[j] == qs[k];
    if (dup || qs[k] >= s.c->n) continue;
    if (!has_rotations_left(s, qr, qs[k])) continue;
    if (cap_pos >= 0 && qr.pos(s, qs[k]) > cap_pos) continue;
    const bool need = ((home >> k) & 1u) || (long)qr.next(s, qs[k]) <= home_next;
    want += need;
    if (take_item(s, qr, qs[k], &r.it[k])) {
      ++items;
      got += need;
      rot += (int)r.it[k].pre.size() + (r.it[k].y >= 0) + (int)r.it[k].post.size();
    }
  }
  if (full && (got < want || items == 0)) {
    s.undo_to(mark);
    return false;
  }
  std::vector<int> cand(s.front.begin(), s.front.end());
  for (int g : cand)
    if (s.c->gates[g].kind == G_CZ && ready(s, g)) {
      s.absorb(g);
      r.czs.push_back(g);
    }
  if (items == 0 && r.czs.empty()) {
    s.undo_to(mark);
    return false;
  }
  if (rr) *rr = std::move(r);
  if (n_rot) *n_rot = rot;
  return true;
}

// strict_catch_up: partial rounds of a multi-tile pass take only qubits at
// the tile's least advanced level (when none of them is ready the pass ends);
// otherwise the level cap rises until some group can take a round.
int run_pass_rounds(Sim& s, const QubitRots& qr, const Tile& t, std::vector<StepRec>* steps, bool allow_partial,
                    bool strict_catch_up) {
  const bool rising = !strict_catch_up || (int)t.local_to_global.size() >= s.c->n;
  int total = 0;
  auto group_qubits = [&](int gi, int (&qs)[4]) {
    for (int k = 0; k < 4; ++k) qs[k] = t.local_to_global[t.groups[gi][k]];
  };
  // home qubits of each group: those not in an earlier group
  std::vector<uint32_t> home(t.groups.size(), 0u);
  for (int gi = 0; gi < (int)t.groups.size(); ++gi)
    for (int k = 0; k < 4; ++k) {
      bool earlier = false;
      for (int gj = 0; gj < gi; ++gj)
        for (int b : t.groups[gj]) earlier |= b == t.groups[gi][k];
      if (!earlier) home[gi] |= 1u << k;
    }
  for (;;) {
    // prefer the group that absorbs the most full rounds (then the most rotations)
    int best = -1, best_rounds = 0, best_rot = 0;
    for (int gi = 0; gi < (int)t.groups.size(); ++gi) {
      int qs[4];
      group_qubits(gi, qs);
      const size_t mark = s.log.size();
      int nr = 0, rot = 0, r1;
      while (nr < kMaxStepRounds && form_round(s, qr, qs, true, nullptr, &r1, home[gi])) {
        ++nr;
        rot += r1;
      }
      s.undo_to(mark);
      if (nr > best_rounds || (nr == best_rounds && rot > best_rot)) {
        best = gi;
        best_rounds = nr;
        best_rot = rot;
      }
    }
    bool partial = false;
    int cap = -1;
    // least and most advanced levels (rotations done) of the tile's qubits
    auto tile_levels = [&](int& lo, int& hi) {
      lo = 1 << 30;
      hi = 0;
      for (int q : t.local_to_global)
        if (q < s.c->n && has_rotations_left(s, qr, q)) {
          lo = std::min(lo, qr.pos(s, q));
          hi = std::max(hi, qr.pos(s, q));
        }
    };
    if (best_rounds == 0) {
      if (!allow_partial) break;
      // no full round anywhere: a partial round of the tile's least
      // advanced qubits (the cap rises until some group can take one), in
      // the group that absorbs most
      int tile_min, tile_max;
      tile_levels(tile_min, tile_max);
      best = -1;
      for (int c = tile_min; c <= (rising ? tile_max : tile_min) && best < 0; ++c) {
        best_rot = -1;
        for (int gi = 0; gi < (int)t.groups.size(); ++gi) {
          int qs[4];
          group_qubits(gi, qs);
          const size_t mark = s.log.size();
          int r1 = 0;
          if (form_round(s, qr, qs, false, nullptr, &r1, home[gi], c) && r1 > best_rot) {
            best = gi;
            best_rot = r1;
            cap = c;
          }
          s.undo_to(mark);
        }
      }
      if (best < 0) break;
      partial = true;
    }
    int qs[4];
    group_qubits(best, qs);
    StepRec st;
    st.group = best;
    const size_t mark = s.log.size();
    for (int nr = 0; nr < kMaxStepRounds; ++nr) {
      RoundRec rr;
      int r1 = 0;
      bool ok = form_round(s, qr, qs, true, &rr, &r1, home[best]);
      if (!ok && partial) {
        // a catch-up round: the first at the cap found above, later ones of
        // qubits at the tile's current least advanced level
        int lo = cap, hi;
        if (nr > 0) tile_levels(lo, hi);
        ok = form_round(s, qr, qs, false, &rr, &r1, home[best], lo);
      }
      if (!ok) break;
      int pads = 0;
      for (int k = 0; k < 4; ++k) pads += rr.it[k].empty();
      total += 4 * r1 - pads;  // useful rotations, minus identity items
      st.rounds.push_back(std::move(rr));
    }
    st.gates.assign(s.log.begin() + mark, s.log.end());
    if (steps) steps->push_back(std::move(st));
  }
  return total;
}

// Candidate tiles for a multi-pass plan: low nibble {0..3} plus K-4 others.
std::vector<std::vector<int>> tile_candidates(const Sim& s, int n_eff, int K) {
  std::vector<std::vector<int>> cands;
  const int extra = K - 4;
  // urgency: qubits whose next pending rotation comes earliest
  std::vector<std::pair<long, int>> urg;
  std::vector<long> next(n_eff, (long)1 << 40);
  for (int g = 0; g < (int)s.done.size(); ++g) {
    if (s.done[g]) continue;
    const Gate& gt = s.c->gates[g];
    if (is_rot(gt.kind) && next[gt.q0] > g) next[gt.q0] = g;
  }
  for (int q = 4; q < n_eff; ++q) urg.push_back({next[q], q});
  std::stable_sort(urg.begin(), urg.end());
  {
    std::vector<int> c = {0, 1, 2, 3};
    for (int i = 0; i < extra; ++i) c.push_back(urg[i].second);
    cands.push_back(c);
  }
  for (int st = 4; st + extra <= n_eff; ++st) {
    std::vector<int> c = {0, 1, 2, 3};
    for (int i = 0; i < extra; ++i) c.push_back(st + i);
    cands.push_back(c);
  }
  // two separate runs of (K-4)/2 qubits each when K-4 is even
  if (extra >= 2 && extra % 2 == 0) {
    int h = extra / 2;
    for (int a = 4; a + h <= n_eff; a += h)
      for (int b = a + h; b + h <= n_eff; b += h) {
        std::vector<int> c = {0, 1, 2, 3};
        for (int i = 0; i < h; ++i) c.push_back(a + i);
        for (int i = 0; i < h; ++i) c.push_back(b + i);
        cands.push_back(c);
      }
  }
  // unions of disjoint 4-qubit chunks, aligned from qubit 4 up ({4k..4k+3})
  // or from the top qubit down ({n-4k..n-4k+3}), so every qubit belongs to
  // some aligned chunk when n is not a multiple of 4 (qubits of one chunk tend
  // to advance together, so round steps on them stay full)
  if (extra % 4 == 0 && extra > 0) {
    std::vector<int> chunks;
    for (int b = 4; b + 4 <= n_eff; b += 4) chunks.push_back(b);
    for (int b = n_eff - 4; b >= 4; b -= 4) chunks.push_back(b);
    std::sort(chunks.begin(), chunks.end());
    chunks.erase(std::unique(chunks.begin(), chunks.end()), chunks.end());
    const int need = extra / 4;
    std::vector<int> pick(need);
    std::function<void(int, int)> rec = [&](int at, int from) {
      if (at == need) {
        std::vector<int> c = {0, 1, 2, 3};
        for (int b : pick)
          for (int k = 0; k < 4; ++k) c.push_back(b + k);
        cands.push_back(c);
        return;
      }
      for (int i = from; i < (int)chunks.size(); ++i) {
        if (at > 0 && chunks[i] < pick[at - 1] + 4) continue;  // disjoint
        pick[at] = chunks[i];
        rec(at + 1, i + 1);
      }
    };
    rec(0, 0);
  }
  for (auto& c : cands) std::sort(c.begin(), c.end());
  std::sort(cands.begin(), cands.end());
  cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
  return cands;
}

inline uint32_t w0(uint32_t code, uint32_t a = 0) { return code | a; }

}  // namespace

void build_hea(Circuit& c, int n, int d, int entangler) {
  if (n < 1 || n > kMaxQubits) throw std::runtime_error("n_qubits must be in 1..30");
  if (d < 0) throw std::runtime_error("n_layers must be >= 0");
  if (entangler != 0 && entangler != 1) throw std::runtime_error("unknown entangler");
  c = Circuit();
  c.n = n;
  c.layers = d;
  c.n_params = 3 * n * d;
  for (int l = 0; l < d; ++l) {
    for (int q = 0; q < n; ++q)
      for (int g = 0; g < 3; ++g)
        c.gates.push_back({g == 1 ? G_RY : G_RZ, q, -1, l * 3 * n + 3 * q + g});
    for (int q = 0; q + 1 < n; ++q) c.gates.push_back({G_CZ, q, q + 1, -1});
    if (entangler == 1 && n > 2) c.gates.push_back({G_CZ, n - 1, 0, -1});
  }
  c.gates_per_layer = d > 0 ? (int)c.gates.size() / d : 0;
}

void validate_circuit(const Circuit& c) {
  if (c.n < 1 || c.n > kMaxQubits) throw std::runtime_error("n_qubits must be in 1..30");
  if (c.n_params < 0) throw std::runtime_error("n_params must be >= 0");
  for (size_t i = 0; i < c.gates.size(); ++i) {
    const Gate& g = c.gates[i];
    const std::string at = " (gate " + std::to_string(i) + ")";
    if (g.q0 < 0 || g.q0 >= c.n) throw std::runtime_error("qubit out of range" + at);
    if (g.kind == G_CZ || g.kind == G_CNOT) {
      if (g.q1 < 0 || g.q1 >= c.n || g.q1 == g.q0) throw std::runtime_error("bad two-qubit target" + at);
    } else if (is_rot(g.kind)) {
      if (g.param < 0 || g.param >= c.n_params) throw std::runtime_error("param out of range" + at);
    } else {
      throw std::runtime_error("unsupported gate kind" + at);
    }
  }
}

int ckpt_interval_gates(const Circuit& c, int ckpt_layers) {
  if (ckpt_layers <= 0) ckpt_layers = 10;
  int per_layer = c.layers > 0 ? c.gates_per_layer : std::max(1, c.n * 4);
  long g = (long)ckpt_layers * per_layer;
  return (int)std::min<long>(g, 1L << 30);
}

// Round programs take RZ, RY and RX rotations and CZs on neighbouring
// qubits, plus the ring's CZ(n-1, 0) when n >= 5 (then qubits 0 and n-1
// never share a register group).
static bool round_eligible(const Circuit& c) {
  for (const Gate& g : c.gates) {
    if (g.kind == G_CNOT) return false;
    if (g.kind != G_CZ) continue;
    const int dq = std::abs(g.q0 - g.q1);
    if (dq != 1 && !(c.n >= 5 && dq == c.n - 1)) return false;
  }
  return true;
}

static void fill_slots(const Circuit& c, std::vector<int32_t>& slot_param, std::vector<int32_t>& slot_kind,
                       std::vector<int32_t>& slot_gate, std::vector<int32_t>& param_off,
                       std::vector<int32_t>& param_slots) {
  for (int g = 0; g < (int)c.gates.size(); ++g)
    if (is_rot(c.gates[g].kind)) {
      slot_param.push_back(c.gates[g].param);
      slot_kind.push_back(c.gates[g].kind);
      slot_gate.push_back(g);
    }
  param_off.assign(c.n_params + 1, 0);
  for (int p : slot_param) param_off[p + 1]++;
  for (int p = 0; p < c.n_params; ++p) param_off[p + 1] += param_off[p];
  param_slots.assign(slot_param.size(), 0);
  std::vector<int32_t> fill(param_off.begin(), param_off.end() - 1);
  for (int s = 0; s < (int)slot_param.size(); ++s) param_slots[fill[slot_param[s]]++] = s;
}

// Checkpoint mode A (Sec. 3.4 with the gradient checkpointing of its memory
// analysis). The forward program is cut into segments at its checkpoints
// (OP_CKPT ops, and pass outputs that are checkpoints); a block is the run of
// segments between two checkpoints. The adjoint, block by block from the
// last: re-run the block's forward segments from the block's input checkpoint
// (psi_0 generated for the first block), storing every segment output but
// the last (which is the next checkpoint, or psi_M), in pass-output slots;
// then run the adjoint segments in reverse, each starting from the stored
// output of the forward segment it undoes. psi is not written back.
static void build_mode_a(FusedPlan& P, bool mem_save) {
  struct Seg {
    int pass;                  // forward pass
    int32_t fb, fe;            // forward op range
    int32_t bb, be;            // adjoint op range
    int32_t end_ckpt;          // slot holding the output (-1: none)
  };
  const int np = (int)P.fwd.size();
  std::vector<Seg> segs;
  for (int p = 0; p < np; ++p) {
    const PassDesc& f = P.fwd[p];
    const PassDesc& b = P.bwd[np - 1 - p];
    std::vector<Seg> fs;
    int32_t at = f.op_begin;
    for (int32_t o = f.op_begin; o < f.op_end; ++o) {
      const uint32_t code = P.fwd_ops[2 * o] & 15u;
      if (code == OP_STEP) {
        // round steps are one op; generic steps are followed by their ops
        if (!P.rounds) o += (int32_t)((P.fwd_ops[2 * o] >> 8) & 0xffffu);
      } else if (code == OP_CKPT) {
        fs.push_back({p, at, o, 0, 0, (int32_t)P.fwd_ops[2 * o + 1]});
        at = o + 1;
      }
    }
    fs.push_back({p, at, f.op_end, 0, 0, f.psi_dst >= 0 ? f.psi_dst : -1});
    // adjoint segments: the same cuts at OP_ANCHOR, in reverse order
    std::vector<std::pair<int32_t, int32_t>> bs;
    at = b.op_begin;
    for (int32_t o = b.op_begin; o < b.op_end; ++o) {
      const uint32_t code = P.bwd_ops[2 * o] & 15u;
      if (code == OP_STEP) {
        if (!P.rounds) o += (int32_t)((P.bwd_ops[2 * o] >> 8) & 0xffffu);
      } else if (code == OP_ANCHOR) {
        bs.push_back({at, o});
        at = o + 1;
      }
    }
    bs.push_back({at, b.op_end});
    if (bs.size() != fs.size()) throw std::runtime_error("internal: mode A segment mismatch");
    for (size_t j = 0; j < fs.size(); ++j) {
      fs[j].bb = bs[fs.size() - 1 - j].first;
      fs[j].be = bs[fs.size() - 1 - j].second;
    }
    for (const Seg& sg : fs) {
      if (sg.fe > sg.fb) {
        segs.push_back(sg);
      } else if (sg.end_ckpt >= 0 && !segs.empty()) {
        // an empty segment: its output is its input
        segs.back().end_ckpt = sg.end_ckpt;
      }
    }
  }
  if (segs.empty()) throw std::runtime_error("internal: mode A without segments");
  if (segs.back().end_ckpt < 0) throw std::runtime_error("internal: mode A without the final state");
  const int32_t H = mem_save ? (PF_SRC_H | PF_DST_H) : 0;
  const int32_t base = mem_save ? 0 : P.n_ckpt;  // pass-output slot numbering
  P.ckpt_mode = 1;
  P.mem_save = mem_save;
  P.n_aslots = 0;
  P.a_sched.clear();
  P.a_dir.clear();
  // blocks: [t0, t1] with segs[t1] ending at a checkpoint
  std::vector<std::pair<int, int>> blocks;
  for (int t = 0, t0 = 0; t < (int)segs.size(); ++t)
    if (segs[t].end_ckpt >= 0) {
      blocks.push_back({t0, t});
      t0 = t + 1;
    }
  bool first = true;
  for (int k = (int)blocks.size() - 1; k >= 0; --k) {
    const int t0 = blocks[k].first, t1 = blocks[k].second;
    P.n_aslots = std::max(P.n_aslots, t1 - t0);
    for (int t = t0; t < t1; ++t) {
      PassDesc d = P.fwd[segs[t].pass];
      d.op_begin = segs[t].fb;
      d.op_end = segs[t].fe;
      d.flags = H & PF_DST_H;
      if (t == t0) {
        d.psi_src = t0 == 0 ? SRC_GENERATE : segs[t0 - 1].end_ckpt;
      } else {
        d.psi_src = base + (t - 1 - t0);
        d.flags |= H & PF_SRC_H;
      }
      d.psi_dst = base + (t - t0);
      d.lam_src = d.lam_dst = BUF_NONE;
      P.a_sched.push_back(d);
      P.a_dir.push_back(0);
    }
    for (int t = t1; t >= t0; --t) {
      PassDesc d = P.bwd[np - 1 - segs[t].pass];
      d.op_begin = segs[t].bb;
      d.op_end = segs[t].be;
      d.flags = 0;
      if (t == t1) {
        d.psi_src = segs[t1].end_ckpt;
      } else {
        d.psi_src = base + (t - t0);
        d.flags |= H & PF_SRC_H;
      }
      d.psi_dst = BUF_NONE;
      d.lam_src = first ? LAM_SEED : LAM_BUF;
      d.lam_dst = (k == 0 && t == t0) ? BUF_NONE : LAM_BUF;
      first = false;
      P.a_sched.push_back(d);
      P.a_dir.push_back(1);
    }
  }
}

namespace {
FusedPlan plan_fused_with(const Circuit& c_in, const PlanRequest& req, bool strict_catch_up);
}

// Relative cost of a plan in round units: a round (one item per register bit
// of a 4096-amplitude tile, forward and adjoint), a step boundary (the
// shared-memory transpose and barrier, about a quarter of a round) and, when
// the state spans several tiles, a pass (streaming the state through the
// SMs once per direction, about two rounds; fitted to GB300 timings of the
// hardware-efficient ansatz at n = 18).
static double plan_cost(const FusedPlan& P) {
  const double passes = P.n_eff > P.K ? (double)P.fwd.size() : 0.0;
  return (double)P.n_rounds + 0.25 * P.n_steps + 2.0 * passes;
}

namespace {
// The circuit with qubit q relabelled (q + s) mod n. Round programs stay
// eligible: a CZ between neighbours q, q+1 (or the ring's n-1, 0) joins
// neighbours again, or the pair n-1, 0.
Circuit shifted(const Circuit& c, int s) {
  if (s == 0) return c;
  Circuit r = c;
  for (Gate& g : r.gates) {
    g.q0 = (g.q0 + s) % c.n;
    if (g.q1 >= 0) g.q1 = (g.q1 + s) % c.n;
  }
  return r;
}
}  // namespace

// Layout and catch-up rule. Every tile holds simulated qubits 0..3 (whole
// 128-byte runs of the state), so a chain whose end sits there is cut into two
// segments by most tiles, and each pass's light cone is shallower. For
// multi-tile round programs the planner therefore tries every cyclic shift
// of the qubits and both catch-up rules (or the one req.catch_up names) on a
// prefix of the circuit (about 16 layers of the ansatz; the plan's structure
// repeats) and keeps the cheapest.
void choose_layout(const Circuit& c, const PlanRequest& req, int* qshift, int* strict) {
  *qshift = 0;
  *strict = req.catch_up > 0 ? 1 : 0;
  Circuit pre = c;
  pre.layers = -1;
  pre.gates.resize(std::min<size_t>(c.gates.size(), (size_t)64 * std::max(c.n, 1)));
  PlanRequest rq = req;
  rq.ckpt_layers = 1 << 30;
  rq.ckpt_mode = 0;
  rq.mem_save = false;
  const FusedPlan probe = plan_fused_with(pre, rq, false);
  if (!probe.rounds || probe.n_eff <= probe.K) return;
  double best = req.catch_up > 0 ? std::numeric_limits<double>::infinity() : plan_cost(probe);
  const int shifts = req.relabel && c.n >= 5 ? c.n : 1;
  for (int s = 0; s < shifts; ++s) {
    const Circuit cs = shifted(pre, s);
    for (int st = 0; st < 2; ++st) {
      if (s == 0 && st == 0) continue;  // the probe
      if (req.catch_up >= 0 && st != req.catch_up) continue;
      const double cost = plan_cost(plan_fused_with(cs, rq, st != 0));
      if (cost < best) {
        best = cost;
        *qshift = s;
        *strict = st;
      }
    }
  }
}

FusedPlan plan_fused(const Circuit& c_in, const PlanRequest& req) {
  int s = req.qshift, st = req.strict;
  if (s < 0 || st < 0) choose_layout(c_in, req, &s, &st);
  if (!req.relabel || c_in.n < 5) s = 0;
  FusedPlan P = plan_fused_with(shifted(c_in, s), req, st != 0);
  P.qshift = s;
  P.strict = st;
  return P;
}

namespace {
FusedPlan plan_fused_with(const Circuit& c_in, const PlanRequest& req, bool strict_catch_up) {
  validate_circuit(c_in);
  FusedPlan P;
  P.n_eff = std::max(c_in.n, kRegBits);
  int K = req.tile_bits > 0 ? req.tile_bits : kMaxTileBits;
  if (K < kRegBits || K > kMaxTileBits) throw std::runtime_error("tile_bits must be in 4..12");
  K = std::min(K, P.n_eff);
  // a multi-pass tile needs at least one qubit beyond the low nibble
  if (P.n_eff > K && K < kRegBits + 1) K = kRegBits + 1;
  P.K = K;
  P.rounds = !req.generic && K >= 7 && round_eligible(c_in);
  const Circuit& c = c_in;
  // gradient terms: generic programs have one per rotation, in circuit order
  std::vector<int> term_of_gate(c.gates.size(), -1);
  P.term_off.assign(1, 0);
  if (!P.rounds) {
    for (int g = 0; g < (int)c.gates.size(); ++g)
      if (is_rot(c.gates[g].kind)) {
        term_of_gate[g] = (int)P.term_kind.size();
        P.term_kind.push_back(c.gates[g].kind);
        P.term_params.push_back(c.gates[g].param);
        P.term_off.push_back((int32_t)P.term_params.size());
        P.term_const.push_back(0.0);
      }
  }

  const int M = (int)c.gates.size();
  Dag dag = build_dag(c);
  Sim sim(c, dag);
  QubitRots qr;
  qr.rots.assign(c.n, {});
  qr.cursor.assign(c.n, 0);
  for (int g = 0; g < M; ++g)
    if (is_rot(c.gates[g].kind)) qr.rots[c.gates[g].q0].push_back(g);
  // Round programs end a pass when no group can take a full round; partial
  // rounds (identity-padded items) are used only when no tile progresses
  // otherwise.
  bool allow_partial = false;
  auto pass_run = [&](const Tile& t, std::vector<StepRec>* steps) {
    return P.rounds ? run_pass_rounds(sim, qr, t, steps, allow_partial, strict_catch_up) : run_pass(sim, t, steps);
  };

  // checkpoint boundaries in gate-sequence positions
  const int G = ckpt_interval_gates(c, req.ckpt_layers);
  long next_ckpt = G;
  int prefix = 0;
  int n_ckpt_slots = 0;

  struct PassRec {
    Tile tile;
    std::vector<StepRec> steps;
    std::vector<int> ckpt_after_step;  // slot written after step i (-1 none)
  };
  std::vector<PassRec> passes;

  while (sim.n_done < M || passes.empty()) {
    Tile tile;
    // one tile covers the state: partial rounds stay in the single pass
    allow_partial = !P.rounds || P.n_eff <= K;
    for (int attempt = 0; attempt < 2; ++attempt) {
      int best_score = 0;
      if (P.n_eff <= K) {
        std::vector<int> all;
        for (int q = 0; q < P.n_eff; ++q) all.push_back(q);
        tile = make_tile(all, K);
        size_t mark = sim.log.size();
        best_score = pass_run(tile, nullptr);
        sim.undo_to(mark);
      } else {
        auto cands = tile_candidates(sim, P.n_eff, K);
        best_score = -1;
        // round programs also try each tile with its qubits grouped by progress
        const int layouts = P.rounds && K % 4 == 0 ? 2 : 1;
        for (int i = 0; i < (int)cands.size(); ++i)
          for (int lay = 0; lay < layouts; ++lay) {
            Tile t = lay == 0 ? make_tile(cands[i], K) : make_tile_by_progress(cands[i], K, sim, qr);
            size_t mark = sim.log.size();
            int sc = pass_run(t, nullptr);
            sim.undo_to(mark);
            if (sc > best_score) {
              best_score = sc;
              tile = t;
            }
          }
      }
      if (best_score > 0 || allow_partial) break;
      allow_partial = true;
    }
    PassRec pr;
    pr.tile = tile;
    pass_run(tile, &pr.steps);
    qr.commit(sim);
    if (pr.steps.empty() && M > 0) throw std::runtime_error("planner made no progress");
    // checkpoints: after a step, once every gate before the next boundary is done
    // (recomputed from the absorption order of this pass)
    {
      std::vector<char> done_now(sim.done.begin(), sim.done.end());
      // roll back this pass's steps to replay them in order
      for (auto it = pr.steps.rbegin(); it != pr.steps.rend(); ++it)
        for (int g : it->gates) done_now[g] = 0;
      pr.ckpt_after_step.assign(pr.steps.size(), -1);
      for (size_t si = 0; si < pr.steps.size(); ++si) {
        for (int g : pr.steps[si].gates) done_now[g] = 1;
        while (prefix < M && done_now[prefix]) ++prefix;
        if (next_ckpt < M && prefix >= next_ckpt && prefix < M) {
          pr.ckpt_after_step[si] = n_ckpt_slots++;
          while (next_ckpt <= prefix) next_ckpt += G;
        }
      }
    }
    passes.push_back(std::move(pr));
    if (M == 0) break;
  }
  // A checkpoint whose boundary falls inside a pass of a multi-pass plan moves
  // to that pass's output: the forward then writes no extra copy, and the
  // adjoint pass that undoes the next forward pass starts from the stored
  // state (re-anchored for free) instead of reloading it in the middle of a
  // pass. The last pass's output is psi_M, and a single-pass plan has no
  // later boundary: there the checkpoints stay after their steps.
  if (P.n_eff > K)
    for (size_t pi = 0; pi + 1 < passes.size(); ++pi) {
      std::vector<int>& ck = passes[pi].ckpt_after_step;
      const int ns = (int)ck.size();
      if (ns == 0 || ck[ns - 1] >= 0) continue;
      for (int si = ns - 2; si >= 0; --si)
        if (ck[si] >= 0) {
          ck[ns - 1] = ck[si];
          ck[si] = -1;
          break;
        }
    }
  const int final_slot = n_ckpt_slots;
  P.n_ckpt = n_ckpt_slots + 1;

  // ---- emit forward and backward programs
  P.fuse_off.assign(1, 0);
  P.n_steps = 0;
  if (P.rounds) P.fuse_off.push_back(0);  // fused entry 0 = identity (empty product)
  using Item = std::vector<std::pair<uint32_t, uint32_t>>;
  auto fuse_of = [&](const std::vector<int>& gates) -> uint32_t {
    if (gates.empty()) return 0u;
    for (int g : gates) P.fuse_gates.push_back({c.gates[g].kind, c.gates[g].param, c.gates[g].angle});
    P.fuse_off.push_back((int32_t)P.fuse_gates.size());
    return (uint32_t)P.fuse_off.size() - 2;
  };
  auto new_term = [&](const std::vector<int>& gates, int kind) -> int32_t {
    if (gates.empty()) return -1;
    const int32_t id = (int32_t)P.term_kind.size();
    P.term_kind.push_back(kind);
    double cst = 0.0;
    for (int g : gates) {
      if (c.gates[g].param >= 0) P.term_params.push_back(c.gates[g].param);
      else cst += c.gates[g].angle;
    }
    P.term_off.push_back((int32_t)P.term_params.size());
    P.term_const.push_back(cst);
    return id;
  };
  // A round step: forward rounds in order; the backward step runs the same
  // rounds in reverse, each one links first, then per item the RZ run and the RY.
  auto emit_round_step = [&](const Tile& tile, const StepRec& st, std::vector<Item>& bwd_items) {
    const std::vector<int>& gl = tile.groups[st.group];
    int gq[4];
    for (int r = 0; r < 4; ++r) gq[r] = tile.local_to_global[gl[r]];
    const uint32_t fr0 = (uint32_t)(P.fwd_rounds.size() / kFwdRoundWords);
    std::vector<std::vector<int32_t>> brs;
    for (const RoundRec& rr : st.rounds) {
      uint32_t links = 0;
      for (int g : rr.czs) {
        const int a = std::min(c.gates[g].q0, c.gates[g].q1), b = std::max(c.gates[g].q0, c.gates[g].q1);
        links ^= 1u << (b == a + 1 ? a : b);  // the ring's CZ(n-1, 0) is link n-1
      }
      uint32_t bbits = 0;
      for (int r = 0; r < 3; ++r)
        if (gq[r + 1] == gq[r] + 1 && ((links >> gq[r]) & 1u)) bbits |= 1u << r;
      std::vector<uint32_t> fw(kFwdRoundWords, 0u);
      std::vector<int32_t> bw(kBwdRoundWords, -1);
      uint32_t rx_mask = 0;  // items whose rotation is an RX
      for (int r = 0; r < 4; ++r) {
        const ItemRec& it = rr.it[r];
        std::vector<int> fg = it.pre;
        if (it.y >= 0) {
          fg.push_back(it.y);
          fg.insert(fg.end(), it.post.begin(), it.post.end());
          bw[r] = new_term(it.post, G_RZ);
          bw[4 + r] = new_term({it.y}, c.gates[it.y].kind);  // an RY or an RX
          if (c.gates[it.y].kind == G_RX) rx_mask |= 1u << r;
        } else {
          bw[r] = new_term(it.pre, G_RZ);
        }
        fw[r] = fuse_of(fg);
      }
      fw[4] = links;
      fw[5] = bbits;
      fw[6] = rx_mask;
      for (int r = 0; r < 8; ++r) fw[8 + r] = (uint32_t)bw[r];  // the items' terms (forward shears)
      bw[8] = (int32_t)links;
      bw[9] = (int32_t)bbits;
      bw[10] = (int32_t)rx_mask;
      bw[11] = 0;
      P.has_rx |= rx_mask != 0;
      P.fwd_rounds.insert(P.fwd_rounds.end(), fw.begin(), fw.end());
      brs.push_back(std::move(bw));
    }
    const uint32_t nr = (uint32_t)st.rounds.size();
    if (nr == 0 || nr > (uint32_t)kMaxStepRounds) throw std::runtime_error("internal: bad round count");
    P.fwd_ops.push_back(w0(OP_STEP, (uint32_t)st.group << 4 | nr << 8));
    P.fwd_ops.push_back(fr0);
    ++P.n_steps;
    P.n_rounds += (int)nr;
    const uint32_t br0 = (uint32_t)(P.bwd_rounds.size() / kBwdRoundWords);
    for (auto it = brs.rbegin(); it != brs.rend(); ++it) P.bwd_rounds.insert(P.bwd_rounds.end(), it->begin(), it->end());
    bwd_items.push_back({{w0(OP_STEP, (uint32_t)st.group << 4 | nr << 8), br0}});
  };
  for (size_t pi = 0; pi < passes.size(); ++pi) {
    const PassRec& pr = passes[pi];
    std::vector<int> global_to_local(P.n_eff, -1);
    for (int lb = 0; lb < K; ++lb) global_to_local[pr.tile.local_to_global[lb]] = lb;

    PassDesc fd{};
    fd.K = K;
    fd.n_groups = (int)pr.tile.groups.size();
    uint32_t tile_mask = 0;
    for (int lb = 0; lb < K; ++lb) {
      fd.gmap[lb] = (uint8_t)pr.tile.local_to_global[lb];
      tile_mask |= 1u << pr.tile.local_to_global[lb];
    }
    fd.outer_mask = (uint32_t)(((1ull << P.n_eff) - 1) & ~(uint64_t)tile_mask);
    for (int gi = 0; gi < fd.n_groups; ++gi)
      for (int r = 0; r < 4; ++r) fd.groups[gi][r] = (uint8_t)pr.tile.groups[gi][r];
    fd.op_begin = (int32_t)(P.fwd_ops.size() / 2);

    // backward ops of this pass are built step by step, then reversed
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> bwd_items;

    const int n_steps = (int)pr.steps.size();
    int trailing_ckpt = -1;
    for (int si = 0; si < n_steps; ++si) {
      const StepRec& st = pr.steps[si];
      if (P.rounds) {
        emit_round_step(pr.tile, st, bwd_items);
      } else {
      const std::vector<int>& gl = pr.tile.groups[st.group];
      auto reg_of = [&](int q) -> uint32_t {
        int lb = global_to_local[q];
        for (int r = 0; r < 4; ++r)
          if (gl[r] == lb) return (uint32_t)r;
        throw std::runtime_error("internal: rotation outside its register group");
      };
      // list scheduling inside the step: fused runs per register, then CZ signs
      std::vector<int> S = st.gates;
      std::sort(S.begin(), S.end());
      auto idx_of = [&](int g) {
        auto it = std::lower_bound(S.begin(), S.end(), g);
        return (it != S.end() && *it == g) ? (int)(it - S.begin()) : -1;
      };
      std::vector<int> lin(S.size(), 0);
      for (int g : S)
        for (int s2 : dag.succ[g]) {
          int j = idx_of(s2);
          if (j >= 0) lin[j]++;
        }
      std::vector<char> fin(S.size(), 0);
      auto finish = [&](int i) {
        fin[i] = 1;
        for (int s2 : dag.succ[S[i]]) {
          int j = idx_of(s2);
          if (j >= 0) lin[j]--;
        }
      };
      std::vector<std::pair<uint32_t, uint32_t>> fops;   // forward ops of the step
      std::vector<std::vector<int>> fruns;               // gates of each OP_U (empty otherwise)
      size_t left = S.size();
      while (left > 0) {
        const size_t before = left;
        for (int r = 0; r < 4; ++r) {
          const int q = pr.tile.local_to_global[gl[r]];
          std::vector<int> run;
          for (;;) {
            int pick = -1;
            for (size_t i = 0; i < S.size(); ++i) {
              if (fin[i] || lin[i] != 0) continue;
              const Gate& gt = c.gates[S[i]];
              if (is_rot(gt.kind) && gt.q0 == q) { pick = (int)i; break; }
            }
            if (pick < 0) break;
            run.push_back(S[pick]);
            finish(pick);
            --left;
          }
          if (!run.empty()) {
            for (int g : run) P.fuse_gates.push_back({c.gates[g].kind, c.gates[g].param, c.gates[g].angle});
            P.fuse_off.push_back((int32_t)P.fuse_gates.size());
            const uint32_t mi = (uint32_t)P.fuse_off.size() - 2;
            fops.push_back({w0(OP_U, reg_of(q) << 4 | mi << 8), 0u});
            fruns.push_back(run);
          }
        }
        uint32_t links = 0;
        std::vector<std::pair<int, int>> others;
        std::vector<int> ready_cz;
        for (size_t i = 0; i < S.size(); ++i) {
          if (fin[i] || lin[i] != 0) continue;
          const Gate& gt = c.gates[S[i]];
          if (gt.kind != G_CZ) continue;
          ready_cz.push_back((int)i);
          int a = std::min(gt.q0, gt.q1), b = std::max(gt.q0, gt.q1);
          if (b == a + 1) links ^= 1u << a;  // the same CZ twice cancels
          else others.push_back({a, b});
        }
        for (int i : ready_cz) {
          finish(i);
          --left;
        }
        if (links) {
          fops.push_back({w0(OP_CHAIN), links});
          fruns.push_back({});
        }
        for (auto& ab : others) {
          fops.push_back({w0(OP_CZ), (uint32_t)ab.first | (uint32_t)ab.second << 8});
          fruns.push_back({});
        }
        for (size_t i = 0; i < S.size(); ++i) {
          if (fin[i] || lin[i] != 0) continue;
          const Gate& gt = c.gates[S[i]];
          if (gt.kind != G_CNOT) continue;
          uint32_t ctl = (uint32_t)gt.q0;
          for (int r = 0; r < 4; ++r)
            if (pr.tile.local_to_global[gl[r]] == gt.q0) ctl = (1u << 8) | (uint32_t)r;
          fops.push_back({w0(OP_CNOT, reg_of(gt.q1) << 4), ctl});
          fruns.push_back({});
          finish((int)i);
          --left;
        }
        if (left == before) throw std::runtime_error("internal: step scheduling stalled");
      }
      // forward: STEP header + ops
      P.fwd_ops.push_back(w0(OP_STEP, (uint32_t)st.group << 4 | (uint32_t)fops.size() << 8));
      P.fwd_ops.push_back(0u);
      for (auto& o : fops) {
        P.fwd_ops.push_back(o.first);
        P.fwd_ops.push_back(o.second);
      }
      ++P.n_steps;
      // backward: reversed ops, fused runs expanded into their rotations
      std::vector<std::pair<uint32_t, uint32_t>> bops;
      uint32_t k = 0;
      for (int oi = (int)fops.size() - 1; oi >= 0; --oi) {
        const uint32_t code = fops[oi].first & 15u;
        if (code == OP_U) {
          const uint32_t r = (fops[oi].first >> 4) & 3u;
          const std::vector<int>& run = fruns[oi];
          for (int j = (int)run.size() - 1; j >= 0; --j) {
            const Gate& gt = c.gates[run[j]];
            const int slot = term_of_gate[run[j]];
            bops.push_back({w0(OP_G, r << 4 | (uint32_t)gt.kind << 6 | k << 8), (uint32_t)slot});
            ++k;
          }
        } else {
          bops.push_back(fops[oi]);
        }
      }
      if (k > (uint32_t)kMaxStepSlots) throw std::runtime_error("internal: step slot overflow");
      std::vector<std::pair<uint32_t, uint32_t>> item;
      item.push_back({w0(OP_STEP, (uint32_t)st.group << 4 | (uint32_t)bops.size() << 8), k});
      item.insert(item.end(), bops.begin(), bops.end());
      bwd_items.push_back(std::move(item));
      }
      // checkpoint after this step
      const int ck = pr.ckpt_after_step[si];
      if (ck >= 0) {
        if (si == n_steps - 1 && pi + 1 < passes.size()) {
          trailing_ckpt = ck;  // the pass output itself becomes the checkpoint
        } else {
          P.fwd_ops.push_back(w0(OP_CKPT));
          P.fwd_ops.push_back((uint32_t)ck);
          bwd_items.push_back({{w0(OP_ANCHOR), (uint32_t)ck}});
        }
      }
    }
    fd.op_end = (int32_t)(P.fwd_ops.size() / 2);
    const bool last = pi + 1 == passes.size();
    fd.psi_src = pi == 0 ? SRC_GENERATE : (P.fwd.back().psi_dst >= 0 ? P.fwd.back().psi_dst : BUF_WORK);
    fd.psi_dst = last ? final_slot : (trailing_ckpt >= 0 ? trailing_ckpt : BUF_WORK);
    fd.flags = last ? PF_EXPECT : 0;
    fd.lam_src = BUF_NONE;
    fd.lam_dst = BUF_NONE;
    P.fwd.push_back(fd);

    // backward program of this pass: the step items in reverse order
    PassDesc bd = fd;
    bd.flags = 0;
    bd.op_begin = (int32_t)(P.bwd_ops.size() / 2);
    for (auto it = bwd_items.rbegin(); it != bwd_items.rend(); ++it)
      for (auto& o : *it) {
        P.bwd_ops.push_back(o.first);
        P.bwd_ops.push_back(o.second);
      }
    bd.op_end = (int32_t)(P.bwd_ops.size() / 2);
    P.bwd.push_back(bd);
  }
  // backward pass order is the reverse of the forward one
  std::reverse(P.bwd.begin(), P.bwd.end());
  const int np = (int)P.bwd.size();
  for (int bi = 0; bi < np; ++bi) {
    const int fi = np - 1 - bi;  // forward pass this backward pass undoes
    const PassDesc& f = P.fwd[fi];
    PassDesc& b = P.bwd[bi];
    b.psi_src = f.psi_dst >= 0 ? f.psi_dst : BUF_WORK;
    b.lam_src = bi == 0 ? LAM_SEED : LAM_BUF;
    const bool last_bwd = fi == 0;
    b.psi_dst = (last_bwd || f.psi_src >= 0) ? BUF_NONE : BUF_WORK;
    b.lam_dst = last_bwd ? BUF_NONE : LAM_BUF;
  }
  // parameter -> terms (a parameter used twice in one term is listed twice)
  P.n_terms = (int)P.term_kind.size();
  P.param_off.assign(c.n_params + 1, 0);
  for (int32_t p : P.term_params) P.param_off[p + 1]++;
  for (int p = 0; p < c.n_params; ++p) P.param_off[p + 1] += P.param_off[p];
  P.param_terms.assign(P.term_params.size(), 0);
  {
    std::vector<int32_t> fill(P.param_off.begin(), P.param_off.end() - 1);
    for (int t = 0; t < P.n_terms; ++t)
      for (int j = P.term_off[t]; j < P.term_off[t + 1]; ++j) P.param_terms[fill[P.term_params[j]]++] = t;
  }
  if (req.ckpt_mode == 1) build_mode_a(P, req.mem_save);
  else if (req.ckpt_mode != 0) throw std::runtime_error("ckpt_mode must be 0 or 1");
  else if (req.mem_save) throw std::runtime_error("mem_save needs ckpt_mode 1");
  return P;
}
}  // namespace

PerGatePlan plan_per_gate(const Circuit& c, const PlanRequest& req) {
  validate_circuit(c);
  PerGatePlan P;
  P.n_eff = std::max(c.n, kRegBits);
  std::vector<int32_t> kinds;
  fill_slots(c, P.slot_param, kinds, P.slot_gate, P.param_off, P.param_slots);
  P.n_slots = (int)P.slot_param.size();
  // checkpoints: copy of the state after gate G-1, 2G-1, ... (then psi_M)
  const int M = (int)c.gates.size();
  const int G = ckpt_interval_gates(c, req.ckpt_layers);
  for (long g = G; g < M; g += G) P.ckpt_after.push_back((int32_t)(g - 1));
  P.n_ckpt = (int)P.ckpt_after.size() + 1;
  return P;
}

}  // namespace qf
