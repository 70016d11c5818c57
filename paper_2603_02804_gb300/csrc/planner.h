// Host-side circuit representation and fusion planner.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "qf_internal.h"

namespace qf {

struct Gate {
  int32_t kind, q0, q1, param;
};

struct Circuit {
  int n = 0;              // qubits as created
  int n_params = 0;
  int layers = -1;        // ansatz depth, -1 for a user gate list
  int gates_per_layer = 0;
  std::vector<Gate> gates;
};

// Result of fusion planning for one circuit.
struct FusedPlan {
  int n_eff = 0;   // simulated qubits (>= 4)
  int K = 0;       // tile bits
  int n_slots = 0; // parametrised gates (gradient slots), numbered in circuit order
  int n_ckpt = 0;  // checkpoint state slots including the final state
  int n_steps = 0;
  std::vector<PassDesc> fwd, bwd;
  std::vector<uint32_t> fwd_ops, bwd_ops;   // 2 words per op
  std::vector<int32_t> fuse_off;            // size n_fused + 1
  std::vector<FuseGate> fuse_gates;
  std::vector<int32_t> slot_param, slot_kind, slot_gate;
  std::vector<int32_t> param_off, param_slots;  // CSR param -> slots
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
};

// Throws std::runtime_error with a message on invalid input.
void build_hea(Circuit& c, int n, int d, int entangler);
void validate_circuit(const Circuit& c);
FusedPlan plan_fused(const Circuit& c, const PlanRequest& req);
PerGatePlan plan_per_gate(const Circuit& c, const PlanRequest& req);
int ckpt_interval_gates(const Circuit& c, int ckpt_layers);

}  // namespace qf
