// Launch interfaces of the CUDA kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "qf_internal.h"

namespace qf {

struct PassArgs {
  PassDesc pd;
  int32_t n_eff;
  int32_t tps_log2;       // log2(tiles per sample) = n_eff - K
  int64_t B;              // samples in this call
  const uint2* ops;       // program of this direction
  const uint4* rounds;    // round records of this direction (round programs)
  const float4* rpar;     // per-round parameters, kRoundPar float4 per round (round programs)
  const float* tcb;       // tensor-core path: per-round 32x32 real blocks, TF32 hi then lo, K-major
  const float4* mats;     // fused 2x2 matrices, 2 float4 each
  const float2* cs;       // (cos, sin) of theta/2 per gradient term (generic programs)
  const float2* enc;      // (cos, sin) of x/2, [B][n_eff]
  const float2* psi_in;   // given initial states [B][2^n_in] (QF_ENC_STATE_IN), else null
  int32_t n_in;           // qubits of the given states (<= n_eff; padding qubits |0>)
  float2* work;           // working state [B][2^n_eff]
  float2* lam;            // adjoint state [B][2^n_eff]
  float2* slots;          // checkpoint states [n_ckpt][slot_stride]
  void* hslots;           // bfloat16 (re, im) pass-output slots [n][slot_stride] (PF_SRC_H / PF_DST_H)
  int64_t slot_stride;    // elements between consecutive checkpoint slots
  uint32_t z_mask;        // observable Z part (global bits)
  uint32_t y_count;       // number of Y factors (phase i^y_count)
  const double* dLdE;     // [B]
  double* e_part;         // [B * tiles per sample]
  double* g_part;         // [B * tiles per sample][n_slots], or [B][n_slots] when g_accum
  int32_t n_slots;
  int32_t g_accum;        // round programs: add the partials of a sample's tiles into one row
  int32_t rx_items;       // round programs with RX items (the RX-capable kernels run them)
  // The pass that computes the expectation may also finish the loss: with
  // done != null, the last CTA to finish sums E from e_part and writes E, the
  // loss and dL/dE as loss_kernel does (done: a CTA counter prep zeroes).
  uint32_t* done;
  double* E;              // [B]
  const float* y;         // labels (MSE)
  double* loss;           // [1]
  double* dLdE_out;       // [B]
  int32_t loss_kind;
  double loss_scale;      // 2 / B
};

// Float64 three-shear parameters of a gradient term (complex128 round
// programs): t = tan(w/4), s = sin(w/2) with w = phi - 2 pi k in (-pi, pi],
// wrap = k & 1 (u(phi) = (-1)^k u(w)).
struct alignas(16) Shear64 {
  double t, s;
  int64_t wrap, pad;
};

// Parameters of one round of a complex128 round program: the shears of the 4
// items' rotations and the round's diagonal as (cos, sin) per register index.
struct RoundPar64 {
  Shear64 rot[4];
  double2 ph[16];
};

// A gradient term of a round record, resolved when the plan is made: its
// angle is c + theta[p0] + theta[p1] (-1: no such parameter); p0 <= -2 marks a
// term of more than two parameters, t = -2 - p0, summed through the CSR maps.
struct RoundTerm {
  int32_t p0, p1;
  double c;
};

struct PrepArgs {
  const float* theta;
  const double* theta64;       // if non-null: float64 parameters (complex128 plans), theta unused
  int32_t n_fused;
  const int32_t* fuse_off;
  const FuseGate* fuse_gates;
  float4* mats;                // may be null (complex128 plans need only mats64)
  double* mats64;              // if non-null: the fused 2x2s in float64 too, 8 doubles each
  int32_t n_terms;
  const int32_t* term_off;     // CSR term -> parameters (angles summed)
  const int32_t* term_params;
  const double* term_const;    // constant part of each term's angle (may be null)
  float2* cs;                  // (cos, sin) of phi/2 per term (generic programs), or
  double2* cs64;               // if non-null instead: (cos, sin) of phi/2 in float64
  const float* x;
  const double* x64;           // if non-null: float64 encoding angles, x unused
  int64_t B;
  int32_t n, n_eff;
  int32_t qshift;              // simulated bit of circuit qubit q: (q + qshift) mod n
  float2* enc;
  double2* enc64;              // if non-null instead of enc: (cos, sin) of x/2 in float64
  // round programs: the parameters of every round gathered in round order
  int32_t n_rpf;               // forward rounds
  const uint4* rpf_src;        // forward round records (fused index per item)
  float4* rpf;                 // [n_rpf][kRoundPar]: rotation shears, then the applied diagonal
  int32_t n_rpb;               // backward rounds
  const uint4* rpb_src;        // backward round records (tz[4], ty[4] terms)
  float4* rpb;                 // [n_rpb][kRoundPar]: rotation shears, then the un-applied diagonal
  RoundPar64* rpf64;           // if non-null instead of rpf / rpb: the same in float64
  RoundPar64* rpb64;           //   (complex128 round programs), [n_rpf] / [n_rpb]
  uint32_t* zero_word;         // if non-null: set to 0 (the forward's CTA counter)
  const RoundTerm* rpf_terms;  // per forward / backward round: its 4 rotation terms, then its
  const RoundTerm* rpb_terms;  //   4 RZ-run terms (-1 terms: no parameter, angle 0)
};

// Table elements of the round parameters (prep work items, kRoundPar per round).
__host__ __device__ inline int64_t round_par_elems(const PrepArgs& a) {
  return (int64_t)kRoundPar * ((int64_t)a.n_rpf + a.n_rpb);
}

struct GradReduceArgs {
  const double* g_part;
  int64_t B;
  int64_t tps;          // partial rows per sample
  int64_t slot_stride;  // elements between consecutive partial rows
  int64_t slot_step;    // elements between consecutive slots of one row
  int32_t n_params;
  const int32_t* param_off;
  const int32_t* param_slots;
  int32_t per_sample;
  double* grad;
  double* scratch;      // stage-1 partials of a two-stage reduction (g_reduce_stages() == 2)
};

// Launches of launch_g_reduce for partial rows per sample `tps` and slot
// step: two (a coalesced stage over row chunks, then the fixed-order sum)
// when a sample has at least kGReduceChunk rows of contiguous slots.
constexpr int kGReduceChunk = 256;
inline int g_reduce_stages(int64_t tps, int64_t slot_step) { return slot_step == 1 && tps >= kGReduceChunk ? 2 : 1; }
// Elements of the stage-1 scratch for B samples.
inline int64_t g_reduce_scratch(int64_t B, int64_t tps, int64_t n_slots) {
  return B * ((tps + kGReduceChunk - 1) / kGReduceChunk) * n_slots;
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t st);
// fwd_ctas: CTAs per SM of the forward round-pass instance (0: 3 when the
// grid exceeds two CTAs per SM, else 2); the adjoint always runs two.
cudaError_t launch_pass(bool bwd, const PassArgs& a, cudaStream_t st, int fwd_ctas = 0);
// Forward pass on the tensor cores (round programs, 12-qubit tiles).
cudaError_t launch_pass_tc(const PassArgs& a, cudaStream_t st);
// Per-round B blocks of the tensor-core path from the float64 fused 2x2s.
cudaError_t launch_tc_tables(const uint4* fwd_rounds, int32_t n_rounds, const double* mats64, float* tcb,
                             cudaStream_t st);
// Observables with X/Y qubits outside the pass's tile: E partials [B][rows]
// and the adjoint seed, each as a full pass over the state.
cudaError_t launch_expect_full(const float2* psi, int n_eff, int64_t B, int64_t rows, uint32_t xm, uint32_t zm,
                               uint32_t yc, double* e_part, cudaStream_t st);
cudaError_t launch_seed_full(const float2* psi, float2* lam, int n_eff, int64_t B, uint32_t xm, uint32_t zm,
                             uint32_t yc, const double* dLdE, cudaStream_t st);
// One bounded wait on an mbarrier nothing arrives at (records a timeout).
cudaError_t bounded_wait_probe(long long limit, cudaStream_t st);
// Read and clear the device error word (1: a bounded wait gave up).
cudaError_t device_status(int32_t* code, cudaStream_t st);
cudaError_t launch_e_reduce(const double* e_part, int64_t B, int tps, double* E, cudaStream_t st);
cudaError_t launch_g_reduce(const GradReduceArgs& a, cudaStream_t st);
cudaError_t launch_loss(int kind, const double* E, const float* y, int64_t B, double* loss, double* dLdE,
                        cudaStream_t st);
// The same with float64 labels (complex128 plans).
cudaError_t launch_loss64(int kind, const double* E, const double* y, int64_t B, double* loss, double* dLdE,
                          cudaStream_t st);
// E from its per-tile partials and the loss in one single-block launch (the
// same E, loss and dL/dE as launch_e_reduce then launch_loss), for batches
// where e_loss_fusable(B, tps).
bool e_loss_fusable(int64_t B, int tps);
cudaError_t launch_e_loss(const double* e_part, int tps, int kind, double* E, const float* y, int64_t B,
                          double* loss, double* dLdE, cudaStream_t st);
cudaError_t launch_e_loss64(const double* e_part, int tps, int kind, double* E, const double* y, int64_t B,
                            double* loss, double* dLdE, cudaStream_t st);

// Opt a kernel in to `smem` bytes of dynamic shared memory on the current
// device, once per device (idempotent; two threads racing on a first launch
// only repeat the call; devices past the table are opted in every time).
struct OptIn {
  std::atomic<bool> done[64] = {};
};
cudaError_t opt_in(const void* fn, size_t smem, OptIn& o);

// ---- complex128 passes --------------------------------------------------------
// Arguments of a complex128 pass: the step programs of PassArgs (generic or
// round programs) with float64 tables and states. The tensor-core path is
// complex64 only.
struct PassArgs64 {
  PassDesc pd;
  int32_t n_eff;
  int32_t tps_log2;       // log2(tiles per sample) = n_eff - K
  int64_t B;
  const uint2* ops;       // program of this direction
  const uint4* rounds;    // round records of this direction (round programs), else null
  const RoundPar64* rpar; // per-round parameters (round programs)
  int32_t rx_items;       // round programs with RX items
  const double2* mats;    // fused 2x2 matrices, 4 double2 each: u00, u01, u10, u11 (generic)
  const double2* cs;      // (cos, sin) of phi/2 per gradient term
  const double2* enc;     // (cos, sin) of x/2, [B][n_eff]
  const double2* psi_in;  // given initial states [B][2^n_in] (QF_ENC_STATE_IN), else null
  int32_t n_in;
  double2* work;          // working state [B][2^n_eff]
  double2* lam;           // adjoint state [B][2^n_eff]
  double2* slots;         // checkpoint states [n_ckpt][slot_stride]
  float2* fslots;         // complex64 pass-output slots (PF_SRC_H / PF_DST_H, memory-saving mode)
  int64_t slot_stride;
  uint32_t z_mask;
  uint32_t y_count;
  const double* dLdE;
  double* e_part;         // [B * tiles per sample]
  double* g_part;         // [B * tiles per sample][n_slots]
  int32_t n_slots;
};
cudaError_t launch_pass64(bool bwd, const PassArgs64& a, cudaStream_t st);
cudaError_t launch_expect_full64(const double2* psi, int n_eff, int64_t B, int64_t rows, uint32_t xm, uint32_t zm,
                                 uint32_t yc, double* e_part, cudaStream_t st);
cudaError_t launch_seed_full64(const double2* psi, double2* lam, int n_eff, int64_t B, uint32_t xm, uint32_t zm,
                               uint32_t yc, const double* dLdE, cudaStream_t st);

// ---- batched persistent launch ------------------------------------------------
// Pointers into the workspace are stored as byte offsets from its base and
// rebased in the kernels; theta/x/y/E/grad are element offsets into the
// caller's concatenated buffers. Plan tables are absolute device pointers.
struct BatchCircuit {
  PassArgs fa, ba;            // forward / backward arguments (pd set per pass)
  const PassDesc* fwd;        // forward passes (observable folded in)
  const PassDesc* bwd;
  int32_t n_fwd, n_bwd;
  int32_t samples_per_item;   // samples of one work item (tiles per CTA when a tile is a sample)
  int32_t loss_kind;          // QF_LOSS_SUM or QF_LOSS_MSE
  double inv_B;
  int64_t theta_off, x_off, sample_off, grad_off;
  PrepArgs prep;              // theta, x relative to the caller buffers; tables ws-relative
  int32_t n_params;
  const int32_t* param_off;   // parameter -> gradient terms
  const int32_t* param_terms;
};

struct BatchItem {
  int32_t c;   // circuit
  int32_t b0;  // first sample
};

struct BatchArgs {
  const BatchCircuit* circ;
  int32_t n_circ;
  const BatchItem* items;
  int32_t n_items;
  int32_t* queue;              // work-queue head (zeroed before each launch)
  char* ws;
  const float* theta;
  const float* x;
  const float* y;
  double* E;
  double* grad;
  double* loss;
  double* lterm;               // per-sample loss terms (workspace)
  const int64_t* prep_off;     // [n_circ + 1]
  const int64_t* grad_out_off; // [n_circ + 1]
  int64_t n_samples;
};

// prep, work-queue reset, persistent forward+adjoint, gradient and loss
// reductions: 4 kernels and one memset on `st`.
cudaError_t launch_batch(const BatchArgs& a, int grid, int64_t prep_total, int64_t n_grad_out, cudaStream_t st);
// Persistent batch kernel grid: two CTAs per SM of the current device.
int batch_grid();
// SMs of the current device (queried once per device; 0 if the query fails).
int device_sms();
// Grid of a grid-strided kernel that wants `want` CTAs: at most 16 per SM.
int64_t stream_grid(int64_t want);

// ---- per-gate comparator ------------------------------------------------------
struct PerGateArgs {
  int32_t n_eff;
  int64_t B;
  float2* psi;          // [B][2^n_eff]
  float2* lam;
  int32_t chunks;       // partial rows per sample
};
cudaError_t pg_encode(const PerGateArgs& a, const float2* enc, cudaStream_t st);
cudaError_t pg_load_states(const PerGateArgs& a, const float2* in, int n_in, cudaStream_t st);
cudaError_t pg_rot(const PerGateArgs& a, int kind, int q, const float2* cs, int slot, cudaStream_t st);
cudaError_t pg_cz(const PerGateArgs& a, int c, int t, bool both, cudaStream_t st);
cudaError_t pg_cnot(const PerGateArgs& a, int c, int t, bool both, cudaStream_t st);
cudaError_t pg_expect(const PerGateArgs& a, uint32_t x_mask, uint32_t z_mask, uint32_t y_count,
                      double* e_part, cudaStream_t st);
cudaError_t pg_seed(const PerGateArgs& a, uint32_t x_mask, uint32_t z_mask, uint32_t y_count,
                    const double* dLdE, cudaStream_t st);
cudaError_t pg_rot_bwd(const PerGateArgs& a, int kind, int q, const float2* cs, int slot, double* g_part,
                       cudaStream_t st);
cudaError_t pg_copy(const float2* src, float2* dst, int64_t n, cudaStream_t st);
int32_t pg_chunks(int32_t n_eff);

// Device address of the fixed scratch block on the current device
// (QF_NOALLOC_MAX_BYTES bytes). Looked up with the device current on every
// call whose stream is not being captured, and cached per device for calls
// made during a capture (which then need an earlier uncaptured call).
cudaError_t noalloc_scratch(cudaStream_t st, void** ptr, size_t* bytes);

}  // namespace qf
