// Internal plan format shared by the host planner and the sm_103a kernels.
//
// A plan is a list of passes. A pass streams every tile of the batched state
// once: a tile is the 2^K amplitudes whose indices differ only in K chosen
// "tile bits" (always including global bits 0..3, so every tile is a set of
// contiguous 128-byte runs). The tile sits in shared memory (XOR-swizzled)
// while a program of steps runs on it. A step loads 16 amplitudes per thread
// whose indices differ in 4 tile bits (the step's register group), applies
// every gate absorbed into the step to those registers, and stores them back.
// This is the gate-fusion of Secs. 3.2-3.3 generalised from "one fused 2x2
// per thread-owned pair" to "a fused program per shared-memory tile".
#pragma once
#include <stdint.h>

namespace qf {

constexpr int kThreads = 256;          // threads per CTA of the pass kernels
constexpr int kRegBits = 4;            // amplitudes per thread per step = 16
constexpr int kMaxTileBits = 12;       // 4096 amplitudes = 32 KiB per state tile
constexpr int kTileAmps = 1 << kMaxTileBits;
constexpr int kMaxStepSlots = 32;      // gradient slots reduced per step (bwd)
constexpr int kMaxQubits = 30;

// gate kinds (match the public QF_GATE_* values)
enum GateKind : int32_t { G_RX = 0, G_RY = 1, G_RZ = 2, G_CZ = 3, G_CNOT = 4 };

// Op words: every op is a uint2 {w0, w1}; the low 4 bits of w0 are the code.
enum OpCode : uint32_t {
  OP_STEP = 1,    // w0: group (bits 4-5), op count of the step (bits 8-23); w1: #grad slots
  OP_U = 2,       // fwd: fused 2x2 on register bit r (bits 4-5), matrix index (bits 8-31)
  OP_G = 3,       // bwd: one rotation, register bit r (4-5), kind (6-7), step slot k (8-15); w1: slot id
  OP_CHAIN = 4,   // CZ(q, q+1) for every bit q set in w1 (diagonal sign)
  OP_CZ = 5,      // CZ(c, t): w1 = c | t << 8
  OP_CKPT = 6,    // fwd: write the tile to checkpoint slot w1
  OP_ANCHOR = 7,  // bwd: reload psi of the tile from checkpoint slot w1
  OP_CNOT = 8,    // CNOT with target register bit (bits 4-5); w1: control register bit | 1 << 8,
                  // or the control's global qubit index (a bit of the thread's base index)
};

// Round programs: a step is OP_STEP {w0: group (bits 4-5) | rounds << 8,
// w1: first round}; every round applies one item per register bit r = 0..3
// and then the CZ links of the round.
//   forward round, kFwdRoundWords words: m[4] (fused 2x2 index per register
//     bit, 0 = identity), links, bbits (links between register bits r, r+1),
//     rx (bit r: item r's rotation is an RX), a pad word, tz[4], ty[4] (the
//     items' gradient terms, as below).
//   backward round, kBwdRoundWords words: tz[4], ty[4] (term of the merged RZ
//     run and of the rotation of each item, -1 = none), links, bbits, rx, a
//     pad word.
// An item is an RZ run alone or a rotation (RY or RX) followed by an RZ run.
// A forward round applies per item the rotation and then the RZ run, then the
// links; a backward step runs its rounds in the order stored, each applying
// the links first, then per item the RZ run and then the rotation (the exact
// reverse).
constexpr int kFwdRoundWords = 16;
constexpr int kBwdRoundWords = 12;
constexpr int kMaxStepRounds = 4;   // 8 gradient values per round
// Parameters of one round of a complex64 round program, in float4: [0, 4) the
// shear parameters (tan(w/4), sin(w/2), wrap parity) of the 4 items'
// rotations; [4, 12) the round's diagonal, i.e. the 4 RZ runs (and the CZ
// links between register bits) merged into one phase per register index j:
// float4 4 + m holds (cos a_j, sin a_j) for j = 2m and 2m + 1, times the
// product of the 4 rotations' wrap signs (the kernels do not read the
// parities themselves). Prep fills
// them as kRoundPar work items per round; complex128 programs hold the same
// in float64 (RoundPar64).
constexpr int kRoundPar = 12;

// Source / destination codes of a pass.
enum : int32_t {
  SRC_GENERATE = -1,  // fwd: build psi_0 = (x) RY(x_q)|0> in place
  BUF_WORK = -2,      // the in-place working state buffer
  BUF_NONE = -3,      // nothing stored
  LAM_SEED = -1,      // bwd: lambda = 2 (dL/dE) O psi from the loaded psi
  LAM_BUF = -2,       // bwd: lambda buffer
};

enum PassFlags : int32_t {
  PF_EXPECT = 1,   // last forward pass: emit <O> partials of each tile
  PF_SRC_H = 2,    // psi_src is a bfloat16 pass-output slot (memory-saving mode)
  PF_DST_H = 4,    // psi_dst is a bfloat16 pass-output slot
};

struct PassDesc {
  int32_t op_begin, op_end;   // op range (uint2 units)
  int32_t psi_src, psi_dst;   // SRC_GENERATE / BUF_WORK / BUF_NONE / slot >= 0
  int32_t lam_src, lam_dst;   // bwd only
  int32_t flags;
  int32_t K;                  // tile bits
  int32_t n_groups;
  uint32_t outer_mask;        // global bits not in the tile
  uint32_t xm_local;          // observable X/Y mask in local tile coordinates
  uint8_t gmap[16];           // local tile bit -> global bit
  uint8_t groups[4][4];       // local bits of register group g, register bit r
};

// Fused 1-qubit op of the forward program: product of gates
// fuse_gate[fuse_off[m] .. fuse_off[m+1]) applied in that order.
struct FuseGate {
  int32_t kind;
  int32_t param;   // theta index, or -1 for a constant angle
  double angle;    // the constant angle when param < 0
};

}  // namespace qf
