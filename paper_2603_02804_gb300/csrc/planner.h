// Host-side circuit representation and fusion planner.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "qf_internal.h"

namespace qf {

struct Gate {
  int32_t kind, q0, q1, param;
  double angle = 0.0;  // constant rotation angle when param < 0 (planner-internal gates only)
};

struct Circuit {
  int n = 0;              // qubits as created
  int n_params = 0;
  int layers = -1;        // ansatz depth, -1 for a user gate list
  int gates_per_layer = 0;
  std::vector<Gate> gates;
};

// Result of fusion planning for one circuit.
//
// A gradient term is one (cos, sin) table entry and one reduced partial:
// in a generic program every rotation is its own term; in a round program a
// run of RZ gates on one qubit with nothing non-diagonal between them is one
// term (they share the value (1/2) Im<lambda|Z|psi> and un-apply as one
// phase), so a term lists the parameters whose angles it sums.
struct FusedPlan {
  int n_eff = 0;    // simulated qubits (>= 4)
  int K = 0;        // tile bits
  bool rounds = false;  // round program (straight-line steps) instead of generic ops
  bool has_rx = false;  // round program with RX items (the RX-capable pass kernels run it)
  int n_terms = 0;  // gradient terms
  int n_ckpt = 0;   // checkpoint state slots including the final state
  int n_steps = 0;
  int n_rounds = 0;
  std::vector<PassDesc> fwd, bwd;
  std::vector<uint32_t> fwd_ops, bwd_ops;   // 2 words per op
  std::vector<uint32_t> fwd_rounds;         // kFwdRoundWords per round
  std::vector<int32_t> bwd_rounds;          // kBwdRoundWords per round
  std::vector<int32_t> fuse_off;            // size n_fused + 1
  std::vector<FuseGate> fuse_gates;
  std::vector<int32_t> term_off, term_params, term_kind;  // CSR term -> params
  std::vector<double> term_const;                         // constant angle of each term
  std::vector<int32_t> param_off, param_terms;            // CSR param -> terms
  // Checkpoint mode. 0 (B): the adjoint passes reverse psi in-kernel and
  // re-anchor at the checkpoints. 1 (A, Sec. 3.4): per checkpoint block the
  // forward passes are re-run from the block's input checkpoint, storing each
  // pass output, and each adjoint pass starts from the stored output of the
  // forward pass it undoes. The A schedule is the adjoint's launch list.
  int ckpt_mode = 0;
  bool mem_save = false;     // A: pass outputs stored as bfloat16 (re, im)
  int n_aslots = 0;          // A: pass-output slots (one block's worth)
  std::vector<PassDesc> a_sched;
  std::vector<uint8_t> a_dir;  // 0: forward program pass, 1: adjoint program pass
  // Layout: circuit qubit q is simulated as bit (q + qshift) mod n of the
  // state index (0 for n < 5). Every table, mask and index of the plan is in
  // simulated bits; observables and encodings are mapped at the boundary.
  int qshift = 0;
  int strict = 0;  // catch-up rule the plan was made with (multi-tile round programs)
};

// Per-gate schedule (the unfused comparator path).
struct PerGatePlan {
  int n_eff = 0;
  int n_slots = 0;
  int n_ckpt = 0;
  std::vector<int32_t> ckpt_after;  // gate index after which slot k is written (-1: none)
  std::vector<int32_t> slot_param, slot_gate;
  std::vector<int32_t> param_off, param_slots;
};

struct PlanRequest {
  int tile_bits = 0;     // 0 = auto
  int ckpt_layers = 10;  // checkpoint interval in layers
  bool generic = false;  // force the generic step program
  int ckpt_mode = 0;     // 0 = B (reverse in-kernel), 1 = A (per-block recompute)
  bool mem_save = false; // A only: bfloat16 pass outputs
  bool relabel = true;   // the planner may simulate the qubits in a cyclically shifted order
  int qshift = -1;       // layout to use (-1: choose), as FusedPlan::qshift
  int strict = -1;       // catch-up rule to use (-1: choose), as FusedPlan::strict
  int catch_up = -1;     // rule the layout search may choose (-1: either, 0: rising, 1: strict)
};

// Throws std::runtime_error with a message on invalid input.
void build_hea(Circuit& c, int n, int d, int entangler);
void validate_circuit(const Circuit& c);
FusedPlan plan_fused(const Circuit& c, const PlanRequest& req);
// The layout (qubit shift) and catch-up rule plan_fused would choose.
void choose_layout(const Circuit& c, const PlanRequest& req, int* qshift, int* strict);
PerGatePlan plan_per_gate(const Circuit& c, const PlanRequest& req);
int ckpt_interval_gates(const Circuit& c, int ckpt_layers);

}  // namespace qf
