/*
 * qfuse: batched state-vector simulation of parametrised quantum circuits
 * with fused forward and fused adjoint-method backward passes, for NVIDIA
 * GB300 (sm_103a).
 *
 * Method: Kawase, "Fast and memory-efficient classical simulation of quantum
 * machine learning via forward and backward gate fusion" (arXiv 2603.02804).
 *   - state and gate application: Sec. 3.1 (qubit i is bit i of the index)
 *   - forward gate fusion: Sec. 3.2
 *   - fused backward with in-register recompute: Sec. 3.3, Eqs. 2-3
 *   - adjoint seed lambda_M = 2 (dL/dE) O psi_M: Eq. 4 with the chain rule
 *   - gradient checkpointing of the state: Sec. 3.4, Eqs. 5-8
 *   - matrix-free Pauli expectation and fused CZ: Appendix B
 *
 * Conventions for every entry point:
 *   - Return value is a qf_status; QF_OK on success. No C++ exception
 *     crosses this boundary. qf_last_error() returns a thread-local message
 *     describing the most recent failure of the calling thread.
 *   - Pointers named *_d are device pointers, *_h host pointers. The library
 *     never frees or takes ownership of caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). All device work of a call is enqueued on it; calls return
 *     without synchronising unless documented otherwise.
 *   - A circuit handle serves one stream at a time. Concurrent calls on the
 *     same handle from several threads are not supported.
 *   - A CUDA error raised by an earlier asynchronous launch surfaces as
 *     QF_ERR_CUDA on a later call.
 */
#ifndef QFUSE_H
#define QFUSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qf_status;
#define QF_OK 0
#define QF_ERR_INVALID_ARG 1  /* a pointer, size or enum is out of range   */
#define QF_ERR_UNSUPPORTED 2  /* valid request this build does not handle  */
#define QF_ERR_WORKSPACE 3    /* workspace too small or plan missing       */
#define QF_ERR_OOM 4          /* a plan-time device allocation failed      */
#define QF_ERR_CUDA 5         /* a CUDA runtime call or launch failed      */
#define QF_ERR_TIMEOUT 6      /* a bounded device-side wait gave up        */

/* Gate kinds. Rotations are u(t) = cos(t/2) I - i sin(t/2) P, P in {X,Y,Z}
 * (Sec. 3.3, gradient step); CZ negates amplitudes whose control and target
 * bits are both 1 (Sec. 3.1). */
#define QF_GATE_RX 0
#define QF_GATE_RY 1
#define QF_GATE_RZ 2
#define QF_GATE_CZ 3
#define QF_GATE_CNOT 4 /* q0 control, q1 target (App. B.1); fused into generic steps */

/* Entangler of the hardware-efficient ansatz. */
#define QF_ENT_CHAIN 0 /* CZ(0,1), CZ(1,2), ..., CZ(n-2,n-1)            */
#define QF_ENT_RING 1  /* the chain plus CZ(n-1, 0)                       */

/* Input encodings (how psi_0 is formed for each sample). */
#define QF_ENC_RY_X 0     /* psi_0 = (x) RY(x_q)|0>, x: float32 [batch][n] angles     */
#define QF_ENC_STATE_IN 1 /* psi_0 given: x is complex64 [batch][2^n] as float32
                             (re, im) pairs, e.g. the random initial states of the
                             paper's measurements (Sec. 4); used as given (the
                             library does not normalise it)                          */

/* Execution paths. */
#define QF_PATH_FUSED 0    /* fused forward / fused adjoint (Secs. 3.2-3.3) */
#define QF_PATH_PER_GATE 1 /* one kernel per gate; the unfused comparator   */

/* Losses understood by qf_loss / qf_train_step. */
#define QF_LOSS_SUM 0 /* L = sum_b E_b (the paper's L = E, Sec. 2.1)       */
#define QF_LOSS_MSE 1 /* L = mean_b (E_b - y_b)^2                          */

/* State precision of a plan (qf_plan_opts.precision). The paper's library
 * runs complex64 or complex128 states; its measurements use complex64
 * (Sec. 4). */
#define QF_PREC_C64 0  /* complex64 states, float32 arithmetic, float32 theta and x:
                          qf_forward, qf_backward, qf_train_step(_host, _noalloc)    */
#define QF_PREC_C128 1 /* complex128 states, float64 arithmetic, float64 theta, x and
                          y: qf_forward64, qf_backward64, qf_train_step64(_host)    */

typedef struct qf_circuit qf_circuit;

/* One gate of a user circuit. q1 is the target of a CZ (-1 otherwise);
 * param indexes theta (-1 for constant gates). */
typedef struct {
  int32_t kind;
  int32_t q0;
  int32_t q1;
  int32_t param;
} qf_gate;

/* Pauli-string observable O = i^{#Y} X^{x_mask} Z^{z_mask}: bit q of x_mask
 * (z_mask) set means an X (Z) factor on qubit q; both bits set is a Y
 * (Y = iXZ, Appendix B.2). Evaluated matrix-free: (O psi)_x =
 * i^{#Y} (-1)^{|(x ^ x_mask) & z_mask|} psi_{x ^ x_mask}. When every X/Y qubit
 * lies in the last pass's tile the expectation and the adjoint seed are fused
 * into the last forward / first adjoint pass; otherwise each is one extra
 * pass over the state. */
typedef struct {
  uint64_t x_mask;
  uint64_t z_mask;
} qf_pauli;

/* Planning options; zero-initialise and set what you need. */
typedef struct {
  int32_t path;        /* QF_PATH_FUSED (default) or QF_PATH_PER_GATE           */
  int32_t tile_bits;   /* fused: qubits per tile, 4..12; 0 = min(n, 12). Circuits
                          wider than the tile need >= 5 (4 is raised to 5)      */
  int32_t ckpt_layers; /* checkpoint interval c in ansatz layers (per-gate: same);
                          0 = 10 layers; a value >= depth keeps only psi_M       */
  int32_t host_only;   /* 1 = build the plan on the host only (no device tables;
                          forward/backward then fail with QF_ERR_WORKSPACE)      */
  int32_t program;     /* fused: 0 = round steps when the circuit allows (RZ/RY
                          rotations, CZ on neighbouring qubits, tile >= 7 qubits),
                          else generic steps; 1 = always generic steps           */
  int32_t ckpt_mode;   /* fused: how the adjoint gets psi_{j-1} (Secs. 3.3-3.4).
                          0 (default): each adjoint pass un-applies the gates to
                          psi in-kernel and re-anchors at the stored checkpoints.
                          1: per checkpoint block, the block's forward passes are
                          re-run from its input checkpoint storing every pass
                          output, and each adjoint pass starts from the stored
                          output of the forward pass it undoes (psi is re-anchored
                          every pass; costs about one extra forward and p*c more
                          stored states, p passes per layer, c layers a block)  */
  int32_t mem_save;    /* ckpt_mode 1 only: store those pass outputs as bfloat16
                          (re, im), computing in float32 (the memory-saving mode
                          of Sec. 3.2); checkpoints and psi_M stay float32       */
  int32_t tc_path;     /* fused: 1 = forward passes (and mode-1 re-runs) apply
                          each round of 4 single-qubit gates as a 32x32 real
                          block on the tensor cores, split-precision 3xTF32 with
                          float32 accumulation; needs round programs and
                          12-qubit tiles (n >= 12), else QF_ERR_UNSUPPORTED.
                          The paper has no tensor-core path (Sec. 3.2 fuses the
                          unitaries, applied here as dense blocks)               */
  int32_t no_host_staging; /* 1: leave out the workspace's host-input staging
                          (x, theta, y and outputs of qf_train_step_host, which
                          then fails); for device-resident inputs of large states */
  int32_t precision;   /* QF_PREC_C64 (default) or QF_PREC_C128. complex128 needs
                          the fused path and runs the same programs (round or
                          generic steps) in float64 on the CUDA cores; tc_path
                          must be 0. With ckpt_mode 1 and
                          mem_save the stored pass outputs are complex64 (float32
                          re, im; the paper's memory-saving mode halves the
                          precision of stored states). Checkpoints, psi_M and
                          all arithmetic stay float64                           */
  int32_t catch_up;    /* fused round programs over several tiles (n > tile_bits):
                          how a pass fills rounds when the qubits of a register
                          group have done different numbers of rotations (the CZ
                          chain lets a qubit run at most one layer ahead of its
                          neighbours). 0 = the planner's choice (both rules and
                          every qubit layout priced on a prefix of the circuit),
                          1 = strict (catch-up rounds take only the tile's least
                          advanced qubits), 2 = rising (the level cap rises until
                          some group can take a round). Tuning knob of Sec. 3.2's
                          fusion grouping; results do not depend on it          */
  int32_t fwd_ctas;    /* fused forward round passes: CTAs per SM the pass kernel
                          is budgeted for (registers per thread): 0 = automatic
                          (3 when a pass has more tiles than two CTAs per SM
                          hold, else 2), 2 or 3. Tuning knob; results do not
                          depend on it                                          */
  int32_t reserved[4];
} qf_plan_opts;

/* Summary of a plan (host-side numbers). */
typedef struct {
  int32_t n_qubits;        /* as created                                       */
  int32_t n_eff;           /* simulated qubits (>= 4: smaller circuits padded)  */
  int32_t n_params;
  int32_t n_slots;         /* gradient slots = parametrised gates               */
  int32_t path;
  int32_t tile_bits;       /* K */
  int32_t n_passes;        /* forward passes (= backward passes)                */
  int32_t n_steps;         /* register steps over all forward passes            */
  int32_t n_fused_ops;     /* fused 2x2 ops of the forward program              */
  int32_t n_ckpt;          /* checkpoint slots incl. the final state            */
  int32_t ckpt_layers;
  int32_t launches_fwd;    /* kernels launched by qf_forward                    */
  int32_t launches_bwd;    /* kernels launched by qf_backward                   */
  int64_t batch;           /* batch the workspace was sized for                 */
  int64_t workspace_bytes;
  int64_t state_bytes;     /* one batched state buffer                          */
  int32_t ckpt_mode;       /* as planned (opts->ckpt_mode)                      */
  int32_t mem_save;
  int32_t n_pass_slots;    /* ckpt_mode 1: stored pass outputs of one block     */
  int32_t tc_path;
  int32_t precision;       /* QF_PREC_C64 or QF_PREC_C128                       */
  int32_t qubit_shift;     /* fused plans: circuit qubit q is simulated as bit
                              (q + qubit_shift) mod n of the state index (the
                              planner's layout; 0 for QF_ENC_STATE_IN circuits).
                              Inputs, observables and results use circuit
                              qubits; only exported programs show the layout  */
  int32_t catch_up;        /* catch-up rule of the plan: 1 strict, 2 rising
                              (0: single-tile or generic programs)             */
  int32_t fwd_ctas;        /* as planned (opts->fwd_ctas)                      */
} qf_plan_info_t;

/* Create the hardware-efficient ansatz of the paper's benchmarks with the
 * gate set of this build: every layer applies RZ, RY, RZ to every qubit and
 * then the entangler (Sec. 4.2 and the ansatz figure; RZ,RY,RZ + CZ chain per
 * layer). `encoding` (QF_ENC_*) forms psi_0: RY(x_q)|0> on every qubit, or a
 * given state. Parameter index of rotation g in {0: first RZ, 1: RY, 2:
 * second RZ} on qubit q of layer l is l*3n + 3q + g, so theta has
 * 3*n*n_layers entries. n_qubits in 1..30, n_layers >= 0. *out receives a new
 * handle (free with qf_circuit_destroy). */
qf_status qf_hea_create(int32_t n_qubits, int32_t n_layers, int32_t entangler, int32_t encoding,
                        qf_circuit** out);

/* Create a circuit from a gate list applied in order after the encoding
 * (Sec. 2.1: U = U_M ... U_1). Supported kinds: QF_GATE_RX/RY/RZ
 * (param in 0..n_params-1; several gates may share a parameter, their
 * gradients add), QF_GATE_CZ and QF_GATE_CNOT (param -1). The gate array is
 * copied.
 * `encoding` as for qf_hea_create. */
qf_status qf_circuit_create(int32_t n_qubits, const qf_gate* gates, int32_t n_gates,
                            int32_t n_params, int32_t encoding, qf_circuit** out);

/* Destroy a handle and the device tables its plan owns. NULL is accepted. */
qf_status qf_circuit_destroy(qf_circuit* c);

/* Plan the circuit for batches of up to `batch` samples (Secs. 3.2-3.4):
 * fuse gates into passes over shared-memory tiles, place checkpoints of the
 * state every opts->ckpt_layers layers, size the workspace, and (unless
 * host_only) upload the plan's device tables. This is the only call that
 * allocates device memory; it may be called again to re-plan.
 * *workspace_bytes receives the size of the caller-allocated workspace that
 * forward/backward/train_step need (256-byte aligned base required). */
qf_status qf_plan(qf_circuit* c, const qf_plan_opts* opts, int64_t batch,
                  size_t* workspace_bytes);

/* The paper's checkpoint memory model (Sec. 3.4, Eqs. 5-8): with checkpoint
 * blocks of b layers, d layers and k state vectors stored per layer of the
 * active block (k = l_var + l_const for per-gate autograd, Eq. 5;
 * k = ceil(l_var / alpha) for fused gates, Eq. 7), peak storage is
 * (k b + d / b) state vectors. Returns that count; *b_best (may be NULL)
 * receives the minimiser sqrt(d / k) (Eqs. 6 and 8). Host only. */
double qf_mem_model(double k, double d, double b, double* b_best);

/* Plan like qf_plan, choosing the checkpoint interval from memory: the
 * smallest interval c (most checkpoints, least reversal drift) whose
 * workspace for `batch` samples fits in mem_bytes. *ckpt_layers receives c
 * (0 and QF_ERR_WORKSPACE when even one checkpoint of psi_M does not fit).
 * opts->ckpt_layers is ignored. */
qf_status qf_plan_fit(qf_circuit* c, const qf_plan_opts* opts, int64_t batch, size_t mem_bytes,
                      int32_t* ckpt_layers, size_t* workspace_bytes);

/* Fill *info with the current plan's summary. */
qf_status qf_plan_info(const qf_circuit* c, qf_plan_info_t* info);

/* Export the forward (direction 0) or backward (1) program for inspection,
 * or (direction 2, ckpt_mode 1 plans) the adjoint's launch list:
 * writes up to cap int32 words to buf (may be NULL) and the full length to
 * *len. Layout: [program kind (0 generic steps, 1 round steps), qubit shift
 * (qf_plan_info_t.qubit_shift: every qubit index and mask below is a
 * simulated bit), n_passes,
 * then per pass: 11 header words (op_begin, op_end, psi_src, psi_dst,
 * lam_src, lam_dst, flags, K, n_groups, outer_mask, xm_local), 16 gmap
 * words, 16 group words], then [n_ops, 2 words per op], then [n_fused, per
 * fused op: count, then count (kind, param, angle as 2 words) gates, param -1
 * for a constant angle], then [n round words of this direction, the words],
 * then [n_terms, per gradient term: kind, count, count parameters, constant
 * angle as 2 words]. Doubles are exported as (low, high) words of their bits. Direction 2: [program kind, qubit shift, n_launches, then per
 * launch: program (0 forward, 1 backward; op ranges index that direction's
 * ops), the 11 header words, 16 gmap words, 16 group words]. Host only. */
qf_status qf_plan_export(const qf_circuit* c, int32_t direction, int32_t* buf,
                         int64_t cap, int64_t* len);

/* Forward expectations E_b = <psi_M|O|psi_M> (Eq. 1) for b < batch.
 * theta_d: float32 [n_params]; x_d: float32 [batch][n_qubits] encoding
 * angles (QF_ENC_RY_X), or the initial states, complex64 [batch][2^n_qubits]
 * (QF_ENC_STATE_IN; qf_backward needs the same x_d); E_d: float64 [batch]
 * (written). The final state and the checkpoints stay in the workspace for a
 * following qf_backward with the same theta, x, batch and observable.
 * batch <= the planned batch. */
qf_status qf_forward(qf_circuit* c, const float* theta_d, const float* x_d, int64_t batch,
                     qf_pauli obs, double* E_d, void* ws_d, size_t ws_bytes, void* stream);

/* Adjoint gradients (Eqs. 2-4) after qf_forward on the same workspace:
 * lambda_M = 2 dLdE_b O psi_M, then gates are un-applied in reverse with
 * dL/dtheta_j = Re<lambda_j| dU_j/dtheta_j |psi_{j-1}> reduced per parameter
 * in float64. dLdE_d: float64 [batch]. grad_d: float64 [n_params] (sum over
 * samples) or [batch][n_params] when per_sample != 0; overwritten. */
qf_status qf_backward(qf_circuit* c, const float* theta_d, const float* x_d, int64_t batch,
                      qf_pauli obs, const double* dLdE_d, double* grad_d, int32_t per_sample,
                      void* ws_d, size_t ws_bytes, void* stream);

/* Loss and dL/dE_b from E (float64 [batch]) and labels y (float32 [batch];
 * ignored for QF_LOSS_SUM, may be NULL then). loss_d: float64 [1];
 * dLdE_d: float64 [batch]. Deterministic single-block reduction. */
qf_status qf_loss(int32_t kind, const double* E_d, const float* y_d, int64_t batch,
                  double* loss_d, double* dLdE_d, void* stream);

/* One training step on device buffers: qf_forward, qf_loss, qf_backward.
 * grad_d: float64 [n_params] = dL/dtheta of the whole batch.
 * Fused plans: from the second consecutive call with the same pointers,
 * sizes, loss and observable, the step's kernels are replayed from a CUDA
 * graph the handle recorded on a stream of its own (the buffers' contents may
 * change between calls; the pointers may not). A call issued while `stream`
 * is being captured by the caller runs its kernels one by one into that
 * capture. With pass timing on (qf_profile), a step replays its graph, timing
 * events included, only when the previous step's timings were read. */
qf_status qf_train_step(qf_circuit* c, const float* theta_d, const float* x_d,
                        const float* y_d, int64_t batch, int32_t loss_kind, qf_pauli obs,
                        double* loss_d, double* E_d, double* grad_d, void* ws_d,
                        size_t ws_bytes, void* stream);

/* The same step from HOST buffers: copies theta_h, x_h (and y_h) into the
 * workspace's staging area, runs the device step, copies loss, E (may be NULL)
 * and grad back, and synchronises `stream` before returning. Pinned host
 * memory gives asynchronous copies; pageable memory works but is slower.
 * Small steps cross the bus as one packed copy each way through a pinned
 * buffer the handle owns. From the second call with the same workspace,
 * batch, loss and observable, that copy-in, the step's kernels and the
 * copy-out are replayed from a CUDA graph the handle recorded (on a stream of
 * its own) instead of being launched one by one; re-planning drops it. The
 * call synchronises, so it cannot itself be captured into a caller's graph. */
qf_status qf_train_step_host(qf_circuit* c, const float* theta_h, const float* x_h,
                             const float* y_h, int64_t batch, int32_t loss_kind, qf_pauli obs,
                             double* loss_h, double* E_h, double* grad_h, void* ws_d,
                             size_t ws_bytes, void* stream);

/* ---- complex128 plans (opts->precision = QF_PREC_C128) ----------------------
 * The same operations as qf_forward, qf_backward, qf_loss, qf_train_step and
 * qf_train_step_host with complex128 states and float64 arithmetic
 * throughout: theta float64 [n_params]; x float64 [batch][n_qubits] angles
 * (QF_ENC_RY_X) or complex128 [batch][2^n_qubits] initial states as float64
 * (re, im) pairs (QF_ENC_STATE_IN); y float64 [batch]. Outputs as for the
 * complex64 calls (float64 E, loss, dL/dE and gradients). Gate tables are
 * computed in float64 and used unrounded. Calling a complex64 entry point on
 * a complex128 plan, or the reverse, returns QF_ERR_INVALID_ARG. */
qf_status qf_forward64(qf_circuit* c, const double* theta_d, const double* x_d, int64_t batch,
                       qf_pauli obs, double* E_d, void* ws_d, size_t ws_bytes, void* stream);
qf_status qf_backward64(qf_circuit* c, const double* theta_d, const double* x_d, int64_t batch,
                        qf_pauli obs, const double* dLdE_d, double* grad_d, int32_t per_sample,
                        void* ws_d, size_t ws_bytes, void* stream);
qf_status qf_loss64(int32_t kind, const double* E_d, const double* y_d, int64_t batch,
                    double* loss_d, double* dLdE_d, void* stream);
qf_status qf_train_step64(qf_circuit* c, const double* theta_d, const double* x_d,
                          const double* y_d, int64_t batch, int32_t loss_kind, qf_pauli obs,
                          double* loss_d, double* E_d, double* grad_d, void* ws_d,
                          size_t ws_bytes, void* stream);
qf_status qf_train_step_host64(qf_circuit* c, const double* theta_h, const double* x_h,
                               const double* y_h, int64_t batch, int32_t loss_kind, qf_pauli obs,
                               double* loss_h, double* E_h, double* grad_h, void* ws_d,
                               size_t ws_bytes, void* stream);

/* Size of the fixed device scratch used by qf_train_step_noalloc. */
#define QF_NOALLOC_MAX_BYTES (32u * 1024u * 1024u)

/* qf_train_step without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * e.g. code embedded in a host application that owns the whole device-memory
 * budget and forbids new allocations after start-up (a real-time control or
 * data-taking loop, a plugin running inside another framework's memory
 * pool), and so can neither call cudaMalloc nor size a workspace per call.
 *
 * Instead of a caller workspace, the step uses one fixed block of device
 * memory of QF_NOALLOC_MAX_BYTES (32 MiB) that the library reserves on every
 * GPU where its device code is loaded and holds until the process exits. The
 * caller still passes inputs and outputs exactly as for qf_train_step
 * (theta_d, x_d, y_d, loss_d, E_d, grad_d: device pointers). The circuit must
 * have been planned with qf_plan; a host_only plan is enough, because this
 * call copies the plan's tables into the fixed block itself. It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * Limits and behaviour:
 *  - complex64 plans only (a complex128 plan returns QF_ERR_INVALID_ARG).
 *  - plan tables plus the step's buffers for `batch` samples must fit in
 *    QF_NOALLOC_MAX_BYTES; otherwise QF_ERR_WORKSPACE is returned and
 *    qf_last_error() states the bytes needed.
 *  - batch must not exceed the batch the circuit was planned for
 *    (QF_ERR_INVALID_ARG otherwise).
 *  - the first call on a device sets it up: it looks up the block's device
 *    address with that device current. Make that first call before any
 *    stream capture. Later calls outside a capture look the address up again
 *    (so a cudaDeviceReset between calls is handled); calls during a capture
 *    reuse the address of the last uncaptured call on that device.
 *  - every call copies the plan's tables from the handle's host memory into
 *    the block, then runs the step there.
 *  - every call shares the one block and it keeps the last call's contents;
 *    each kernel writes every scratch element it later reads, so nothing needs
 *    clearing. Calls that overlap on the GPU (other streams, other threads)
 *    race on the block: serialise them. */
qf_status qf_train_step_noalloc(qf_circuit* c, const float* theta_d, const float* x_d,
                                const float* y_d, int64_t batch, int32_t loss_kind, qf_pauli obs,
                                double* loss_d, double* E_d, double* grad_d, void* stream);

/* Kernels launched by the most recent qf_forward + qf_backward (+ qf_loss
 * inside qf_train_step) on this handle; for launch accounting. */
qf_status qf_launch_count(const qf_circuit* c, int64_t* launches);

/* How many train steps (qf_train_step, qf_train_step64 and the host-buffer
 * steps) this handle recorded as CUDA graphs and how many it replayed from
 * one since it was created; for checking that a training loop hits the
 * replay path (the same buffers, batch, loss and observable every step). */
qf_status qf_graph_stats(const qf_circuit* c, int64_t* recorded, int64_t* replayed);

/* ---- batched launch over many circuits ----------------------------------
 * Many circuits of different widths, depths and batch sizes, trained in one
 * persistent kernel launch: each work item (one sample, or a group of small
 * samples, of one circuit) is taken by one CTA from a work queue ordered
 * largest first, and that CTA runs the item's fused forward passes, its
 * dL/dE and its fused adjoint passes (Secs. 3.2-3.3) with no waits on other
 * CTAs. The loss is summed over every circuit; each circuit gets its own
 * gradient. Per step: 4 kernels and one memset; capturable in a CUDA graph. */
typedef struct qf_batch qf_batch;

/* Build a batched launch. circuits[i] must be planned with QF_PATH_FUSED as
 * round programs (qf_plan_info: tile_bits >= 7, RZ/RY rotations, CZ on
 * neighbouring qubits; host_only plans are fine); batch[i] >= 1 samples of
 * circuit i; obs[i] its observable; loss_kind QF_LOSS_SUM or QF_LOSS_MSE
 * (mean over each circuit's samples, summed over circuits). Allocates the
 * batch's device tables; the circuits must outlive the batch and not be
 * re-planned. *workspace_bytes: size of the caller workspace. */
qf_status qf_batch_create(int32_t n_circuits, qf_circuit* const* circuits, const int64_t* batch,
                          const qf_pauli* obs, int32_t loss_kind, size_t* workspace_bytes,
                          qf_batch** out);

/* Element offsets of each circuit in the concatenated buffers ([n + 1] each,
 * any may be NULL): theta_off (float32 parameters; also float64 gradients),
 * x_off (float32 [B_i][n_i] encodings), sample_off (E and y per sample). */
qf_status qf_batch_layout(const qf_batch* b, int64_t* theta_off, int64_t* x_off, int64_t* sample_off);

/* One training step of every circuit: theta_d, x_d, y_d (MSE only) are the
 * concatenated inputs, E_d (float64 per sample), grad_d (float64 per
 * parameter, dL/dtheta) and loss_d (float64 [1]) are written. */
qf_status qf_batch_train_step(qf_batch* b, const float* theta_d, const float* x_d, const float* y_d,
                              double* loss_d, double* E_d, double* grad_d, void* ws_d, size_t ws_bytes,
                              void* stream);

/* Capture one qf_batch_train_step with these buffers into a CUDA graph owned
 * by the batch (runs one eager step first, then captures on `stream`, which
 * must not be the legacy default stream). qf_batch_graph_launch replays it. */
qf_status qf_batch_graph_capture(qf_batch* b, const float* theta_d, const float* x_d, const float* y_d,
                                 double* loss_d, double* E_d, double* grad_d, void* ws_d,
                                 size_t ws_bytes, void* stream);
qf_status qf_batch_graph_launch(qf_batch* b, void* stream);

/* Work items, total samples and total parameters of the batch. */
qf_status qf_batch_info(const qf_batch* b, int64_t* n_items, int64_t* n_samples, int64_t* n_params);

/* Free the batch's device tables and graph. NULL is accepted. */
qf_status qf_batch_destroy(qf_batch* b);

/* Start (on != 0) or stop timing the pass kernels of the following
 * qf_forward / qf_backward calls on this handle: a CUDA event pair is
 * recorded on the call's stream around the forward passes and around the
 * backward passes (up to 4096 pairs are kept between reads). Starting
 * creates the events (no device memory). */
qf_status qf_profile(qf_circuit* c, int32_t on);

/* Sum of the recorded forward / backward pass-kernel time in milliseconds
 * and the number of pass-kernel launches they cover, since the last read.
 * Waits for the recorded events; resets the counters. Any output may be
 * NULL. */
qf_status qf_profile_read(qf_circuit* c, double* fwd_ms, int64_t* fwd_launches, double* bwd_ms,
                          int64_t* bwd_launches);

/* Read and clear the device error word after the work queued on `stream`
 * (synchronises the stream). *code: 0 = no error; 1 = a bounded wait inside
 * a kernel gave up (the tensor-core path waits on its MMA completions with an
 * iteration limit instead of spinning forever; results of that launch are
 * invalid). Has no counterpart in the paper. */
qf_status qf_device_status(void* stream, int32_t* code);

/* Check of the failure path of the bounded waits: launches one thread that
 * waits on an mbarrier nothing arrives at, gives up after `spin_limit` polls
 * (1..2^20, well under a second) and records the timeout in the device error
 * word; a following qf_device_status then reports 1 and the context stays
 * usable. No paper counterpart. */
qf_status qf_check_bounded_wait(void* stream, int64_t spin_limit);

/* Thread-local description of the last error ("" if none). */
const char* qf_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t qf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QFUSE_H */
