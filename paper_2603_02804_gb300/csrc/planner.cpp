// Fusion planner: turns a gate list into passes over shared-memory tiles.
//
// Forward fusion (Sec. 3.2) is generalised from "consecutive gates on the
// same or adjacent qubits" to "every gate whose dependencies are met and whose
// qubit lies in the current 4-qubit register group", with diagonal gates
// (RZ, CZ) allowed to commute past each other. The backward program is the
// exact reverse of the forward one, with each fused 2x2 expanded back into
// its rotations so every parameter gets its own gradient term (Sec. 3.3).
#include "planner.h"

#include <algorithm>
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
    int qs[2] = {gt.q0, gt.kind == G_CZ ? gt.q1 : -1};
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

struct StepRec {
  int group;
  std::vector<int> gates;
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
    if (steps) steps->push_back({best, std::move(gs)});
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
    if (g.kind == G_CZ) {
      if (g.q1 < 0 || g.q1 >= c.n || g.q1 == g.q0) throw std::runtime_error("bad CZ target" + at);
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

FusedPlan plan_fused(const Circuit& c, const PlanRequest& req) {
  validate_circuit(c);
  FusedPlan P;
  P.n_eff = std::max(c.n, kRegBits);
  int K = req.tile_bits > 0 ? req.tile_bits : kMaxTileBits;
  if (K < kRegBits || K > kMaxTileBits) throw std::runtime_error("tile_bits must be in 4..12");
  K = std::min(K, P.n_eff);
  // a multi-pass tile needs at least one qubit beyond the low nibble
  if (P.n_eff > K && K < kRegBits + 1) K = kRegBits + 1;
  P.K = K;
  fill_slots(c, P.slot_param, P.slot_kind, P.slot_gate, P.param_off, P.param_slots);
  P.n_slots = (int)P.slot_param.size();
  std::vector<int> slot_of_gate(c.gates.size(), -1);
  for (int s = 0; s < P.n_slots; ++s) slot_of_gate[P.slot_gate[s]] = s;

  const int M = (int)c.gates.size();
  Dag dag = build_dag(c);
  Sim sim(c, dag);

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
    if (P.n_eff <= K) {
      std::vector<int> all;
      for (int q = 0; q < P.n_eff; ++q) all.push_back(q);
      tile = make_tile(all, K);
    } else {
      auto cands = tile_candidates(sim, P.n_eff, K);
      int best = -1, best_score = -1;
      for (int i = 0; i < (int)cands.size(); ++i) {
        Tile t = make_tile(cands[i], K);
        size_t mark = sim.log.size();
        int sc = run_pass(sim, t, nullptr);
        sim.undo_to(mark);
        if (sc > best_score) {
          best_score = sc;
          best = i;
        }
      }
      tile = make_tile(cands[best], K);
    }
    PassRec pr;
    pr.tile = tile;
    run_pass(sim, tile, &pr.steps);
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
  const int final_slot = n_ckpt_slots;
  P.n_ckpt = n_ckpt_slots + 1;

  // ---- emit forward and backward programs
  P.fuse_off.assign(1, 0);
  P.n_steps = 0;
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
              if (gt.kind != G_CZ && gt.q0 == q) { pick = (int)i; break; }
            }
            if (pick < 0) break;
            run.push_back(S[pick]);
            finish(pick);
            --left;
          }
          if (!run.empty()) {
            for (int g : run) P.fuse_gates.push_back({c.gates[g].kind, c.gates[g].param});
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
            const int slot = slot_of_gate[run[j]];
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
  return P;
}

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
