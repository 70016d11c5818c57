// C-ABI of the library (declared in include/qfuse.h).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <exception>
#include <map>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "kernels.h"
#include "planner.h"
#include "qfuse.h"

namespace {

thread_local std::string g_err;

qf_status fail(qf_status s, const std::string& m) {
  g_err = m;
  return s;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t theta = 0, x = 0, y = 0, E = 0, dLdE = 0, grad = 0, loss = 0;  // staging
  size_t mats = 0, cs = 0, enc = 0;
  size_t rpf = 0, rpb = 0;  // round-ordered item parameters (round programs)
  size_t mats64 = 0, tcb = 0;  // tensor-core path: float64 fused 2x2s, per-round B blocks
  size_t work = 0, lam = 0, slots = 0, hslots = 0;
  size_t epart = 0, gpart = 0, gred = 0;  // gred: stage-1 scratch of a two-stage gradient reduction
  size_t done = 0;                         // CTA counter of a forward pass that finishes the loss
  size_t total = 0;
  int64_t state_elems = 0;  // batch * 2^n_eff
  int64_t rows = 0;         // partial rows per sample (tiles or chunks)
};

// Plan tables on the device.
struct DevTables {
  const uint2* fwd_ops = nullptr;
  const uint2* bwd_ops = nullptr;
  const int32_t* fuse_off = nullptr;
  const qf::FuseGate* fuse_gates = nullptr;
  const uint4* fwd_rounds = nullptr;
  const uint4* bwd_rounds = nullptr;
  const int32_t* term_off = nullptr;      // CSR term -> parameters
  const int32_t* term_params = nullptr;
  const double* term_const = nullptr;     // constant part of each term's angle (fused plans)
  const int32_t* param_off = nullptr;     // CSR parameter -> terms
  const int32_t* param_terms = nullptr;
  const qf::RoundTerm* fwd_rterms = nullptr;  // round programs: each round's terms, resolved
  const qf::RoundTerm* bwd_rterms = nullptr;
};

// Byte offsets of each table inside the blob.
struct BlobOffsets {
  size_t fwd = 0, bwd = 0, foff = 0, fg = 0, frd = 0, brd = 0, to = 0, tp = 0, tcst = 0, po = 0, ps = 0;
  size_t frt = 0, brt = 0;
};

}  // namespace

// A train step recorded as a CUDA graph for one argument key (pointers,
// sizes, loss and observable).
struct StepGraph {
  std::array<uint64_t, 12> key{};
  bool profile = false;  // recorded with pass-timing events (qf_profile)
  cudaGraphExec_t exec = nullptr;
  bool seen = false;    // the key ran eagerly once
  bool failed = false;  // recording failed for the key: it stays eager
  int64_t launches = 0;
  // timing-event pairs 0 .. ev_pairs-1 recorded by every replay, with their
  // direction and launch counts
  size_t ev_pairs = 0;
  std::vector<int> ev_dir;
  std::vector<int64_t> ev_launches;
};

struct qf_circuit {
  qf::Circuit circ;
  bool planned = false;
  bool host_only = false;
  int path = QF_PATH_FUSED;
  int ckpt_layers = 10;
  int encoding = QF_ENC_RY_X;
  bool staging = true;      // workspace holds host-input staging (qf_train_step_host)
  bool tc = false;          // forward rounds on the tensor cores
  bool f64 = false;         // complex128 states (QF_PREC_C128)
  // layout chosen by the planner for (tile_bits option, program option); kept
  // so that re-planning (e.g. qf_plan_fit's search) does not search again
  bool lay_valid = false;
  int lay_tile_bits = 0, lay_generic = 0, lay_catch_up = 0, lay_shift = 0, lay_strict = 0;
  int fwd_ctas = 0;         // forward round passes: CTAs per SM of the kernel instance (0: automatic)
  int64_t batch = 0;
  qf::FusedPlan fp;
  qf::PerGatePlan gp;
  Layout L;
  std::vector<char> blob;   // host image of the plan's device tables
  BlobOffsets bo;
  void* d_tables = nullptr; // device copy of blob (qf_plan)
  DevTables dt;
  int64_t launches = 0;
  void* h_stage = nullptr;  // pinned host staging of the host-buffer step (packed copies)
  size_t h_stage_bytes = 0;
  // CUDA graphs of the train steps: the host-buffer step's device part
  // (packed copy in, step, packed copy out) and the device-buffer step, each
  // recorded on g_stream for an argument key seen before and replayed on the
  // caller's stream
  cudaStream_t g_stream = nullptr;
  StepGraph hg, dg;
  bool recording = false;  // a step is being recorded on g_stream
  int64_t g_recorded = 0, g_replayed = 0;
  int64_t call_launches = 0;
  // pass-kernel timing (qf_profile)
  bool profile = false;
  std::vector<cudaEvent_t> ev;          // 2 per record
  std::vector<int> ev_dir;              // 0 fwd, 1 bwd
  std::vector<int64_t> ev_launches;
  size_t ev_used = 0;
};

namespace {

constexpr size_t kMaxProfilePairs = 4096;

void destroy_events(qf_circuit* c) {
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  c->ev_dir.clear();
  c->ev_launches.clear();
  c->ev_used = 0;
}

// A timing event; while a step is being recorded it becomes an event-record
// node of the graph (every replay records it).
void record_event(const qf_circuit* c, cudaEvent_t e, cudaStream_t st) {
  if (c->recording) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
}

// Record the start of a timed range; returns the pair index or -1.
int prof_begin(qf_circuit* c, cudaStream_t st) {
  if (!c->profile || c->ev_used >= kMaxProfilePairs) return -1;
  const size_t k = c->ev_used++;
  record_event(c, c->ev[2 * k], st);
  return (int)k;
}

void prof_end(qf_circuit* c, int k, int dir, int64_t launches, cudaStream_t st) {
  if (k < 0) return;
  record_event(c, c->ev[2 * k + 1], st);
  c->ev_dir[k] = dir;
  c->ev_launches[k] = launches;
}

void drop_graph(StepGraph& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G = StepGraph();
}

void free_tables(qf_circuit* c) {
  drop_graph(c->hg);
  drop_graph(c->dg);
  if (c->d_tables) cudaFree(c->d_tables);
  c->d_tables = nullptr;
  c->dt = DevTables();
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
  c->h_stage_bytes = 0;
}

int n_eff_of(const qf_circuit* c) { return c->path == QF_PATH_FUSED ? c->fp.n_eff : c->gp.n_eff; }
// Bytes of one batch of inputs: angles [B][n] float32 (float64), or states
// [B][2^n] complex64 (complex128 plans: complex128).
size_t x_bytes(const qf_circuit* c, int64_t B) {
  const size_t w = c->f64 ? 2 : 1;
  return c->encoding == QF_ENC_STATE_IN ? (size_t)B * ((size_t)1 << c->circ.n) * 8 * w
                                        : (size_t)B * c->circ.n * 4 * w;
}

int n_slots_of(const qf_circuit* c) { return c->path == QF_PATH_FUSED ? c->fp.n_terms : c->gp.n_slots; }

Layout make_layout(const qf_circuit* c, int64_t B) {
  Layout L;
  const int n_eff = n_eff_of(c);
  const int64_t dim = 1ll << n_eff;
  const int P = c->circ.n_params;
  const int S = n_slots_of(c);
  L.state_elems = B * dim;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += al(bytes);
    return at;
  };
  const int64_t Bs = c->staging ? B : 0;  // staged inputs of the host-buffer step
  const size_t rw = c->f64 ? 8 : 4;        // bytes of a real input (theta, y)
  const size_t aw = c->f64 ? 16 : 8;       // bytes of an amplitude
  L.theta = take((size_t)P * rw);
  L.x = take(x_bytes(c, Bs));
  L.y = take((size_t)B * rw);
  L.E = take((size_t)B * 8);
  L.dLdE = take((size_t)B * 8);
  L.grad = take((size_t)P * 8);
  L.loss = take(8);
  L.done = take(4);
  L.cs = take((size_t)S * 16);  // (cos, sin) per term, float32 or float64 (generic programs)
  L.enc = take((size_t)B * n_eff * aw);
  L.work = take((size_t)L.state_elems * aw);
  L.lam = take((size_t)L.state_elems * aw);
  if (c->path == QF_PATH_FUSED) {
    const int n_fused = (int)c->fp.fuse_off.size() - 1;
    if (c->f64) L.mats64 = take((size_t)std::max(n_fused, 0) * 64);
    else L.mats = take((size_t)std::max(n_fused, 0) * 32);
    if (c->fp.rounds) {
      // per round: kRoundPar float4 (complex64) or one RoundPar64 (complex128)
      const size_t per = c->f64 ? sizeof(qf::RoundPar64) : qf::kRoundPar * 16;
      L.rpf = take(c->fp.fwd_rounds.size() / qf::kFwdRoundWords * per);
      L.rpb = take(c->fp.bwd_rounds.size() / qf::kBwdRoundWords * per);
    }
    if (c->tc) {
      L.mats64 = take((size_t)std::max(n_fused, 0) * 64);
      L.tcb = take(c->fp.fwd_rounds.size() / qf::kFwdRoundWords * 2048 * 4);
    }
    // checkpoint mode A: pass-output slots after the checkpoints, or an array
    // of them at half the state's precision (memory-saving mode: bfloat16
    // pairs for complex64 states, complex64 for complex128)
    const int extra = c->fp.ckpt_mode == 1 && !c->fp.mem_save ? c->fp.n_aslots : 0;
    L.slots = take((size_t)(c->fp.n_ckpt + extra) * L.state_elems * aw);
    if (c->fp.ckpt_mode == 1 && c->fp.mem_save) L.hslots = take((size_t)c->fp.n_aslots * L.state_elems * aw / 2);
    L.rows = 1ll << (c->fp.n_eff - c->fp.K);
  } else {
    L.slots = take((size_t)c->gp.ckpt_after.size() * L.state_elems * 8);
    L.rows = qf::pg_chunks(n_eff);
  }
  L.epart = take((size_t)B * L.rows * 8);
  L.gpart = take((size_t)B * L.rows * S * 8);
  if (c->path == QF_PATH_FUSED && qf::g_reduce_stages(L.rows, 1) == 2)
    L.gred = take((size_t)qf::g_reduce_scratch(B, L.rows, S) * 8);
  L.total = o;
  return L;
}

template <class T>
size_t push_table(std::vector<char>& blob, const std::vector<T>& v) {
  size_t at = al(blob.size());
  blob.resize(at + al(std::max<size_t>(v.size() * sizeof(T), 1)));
  if (!v.empty()) memcpy(blob.data() + at, v.data(), v.size() * sizeof(T));
  return at;
}

// The terms of every round record (rotation terms, then RZ-run terms), each
// with its parameters and constant resolved, so that prep reads a round's
// angles without walking the term maps.
template <class W>
std::vector<qf::RoundTerm> round_terms(const qf::FusedPlan& P, const std::vector<W>& rounds, int words,
                                       int tz_at, int ty_at) {
  std::vector<qf::RoundTerm> out;
  const size_t n_rounds = rounds.size() / (size_t)words;
  out.reserve(n_rounds * 8);
  auto ref = [&](int32_t t) {
    qf::RoundTerm e{-1, -1, 0.0};
    if (t < 0) return e;
    const int b0 = P.term_off[t], b1 = P.term_off[t + 1];
    e.c = P.term_const.empty() ? 0.0 : P.term_const[t];
    if (b1 - b0 > 2) {
      e.p0 = -2 - t;
      e.c = 0.0;
      return e;
    }
    if (b1 > b0) e.p0 = P.term_params[b0];
    if (b1 > b0 + 1) e.p1 = P.term_params[b0 + 1];
    return e;
  };
  for (size_t r = 0; r < n_rounds; ++r) {
    const int32_t* rec = reinterpret_cast<const int32_t*>(rounds.data()) + r * words;
    for (int k = 0; k < 4; ++k) out.push_back(ref(rec[ty_at + k]));
    for (int k = 0; k < 4; ++k) out.push_back(ref(rec[tz_at + k]));
  }
  return out;
}

// Serialise the plan's device tables into c->blob (host memory).
void build_blob(qf_circuit* c) {
  std::vector<char>& blob = c->blob;
  blob.clear();
  BlobOffsets& o = c->bo;
  o = BlobOffsets();
  if (c->path == QF_PATH_FUSED) {
    o.fwd = push_table(blob, c->fp.fwd_ops);
    o.bwd = push_table(blob, c->fp.bwd_ops);
    o.foff = push_table(blob, c->fp.fuse_off);
    o.fg = push_table(blob, c->fp.fuse_gates);
    o.frd = push_table(blob, c->fp.fwd_rounds);
    o.brd = push_table(blob, c->fp.bwd_rounds);
    o.to = push_table(blob, c->fp.term_off);
    o.tp = push_table(blob, c->fp.term_params);
    o.tcst = push_table(blob, c->fp.term_const);
    o.po = push_table(blob, c->fp.param_off);
    o.ps = push_table(blob, c->fp.param_terms);
    if (c->fp.rounds) {
      o.frt = push_table(blob, round_terms(c->fp, c->fp.fwd_rounds, qf::kFwdRoundWords, 8, 12));
      o.brt = push_table(blob, round_terms(c->fp, c->fp.bwd_rounds, qf::kBwdRoundWords, 0, 4));
    }
  } else {
    std::vector<int32_t> toff(c->gp.n_slots + 1);
    for (int t = 0; t <= c->gp.n_slots; ++t) toff[t] = t;
    o.to = push_table(blob, toff);
    o.tp = push_table(blob, c->gp.slot_param);
    o.po = push_table(blob, c->gp.param_off);
    o.ps = push_table(blob, c->gp.param_slots);
  }
  blob.resize(al(std::max<size_t>(blob.size(), 1)));
}

// Table pointers for a device copy of c->blob starting at base.
DevTables tables_at(const qf_circuit* c, void* base) {
  char* b = static_cast<char*>(base);
  DevTables t;
  if (c->path == QF_PATH_FUSED) {
    t.fwd_ops = reinterpret_cast<const uint2*>(b + c->bo.fwd);
    t.bwd_ops = reinterpret_cast<const uint2*>(b + c->bo.bwd);
    t.fuse_off = reinterpret_cast<const int32_t*>(b + c->bo.foff);
    t.fuse_gates = reinterpret_cast<const qf::FuseGate*>(b + c->bo.fg);
    t.fwd_rounds = reinterpret_cast<const uint4*>(b + c->bo.frd);
    t.bwd_rounds = reinterpret_cast<const uint4*>(b + c->bo.brd);
    t.term_const = reinterpret_cast<const double*>(b + c->bo.tcst);
    if (c->fp.rounds) {
      t.fwd_rterms = reinterpret_cast<const qf::RoundTerm*>(b + c->bo.frt);
      t.bwd_rterms = reinterpret_cast<const qf::RoundTerm*>(b + c->bo.brt);
    }
  }
  t.term_off = reinterpret_cast<const int32_t*>(b + c->bo.to);
  t.term_params = reinterpret_cast<const int32_t*>(b + c->bo.tp);
  t.param_off = reinterpret_cast<const int32_t*>(b + c->bo.po);
  t.param_terms = reinterpret_cast<const int32_t*>(b + c->bo.ps);
  return t;
}

qf_status upload(qf_circuit* c) {
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, c->blob.size());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(QF_ERR_OOM, std::string("cudaMalloc of plan tables failed: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(d, c->blob.data(), c->blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return fail(QF_ERR_CUDA, std::string("plan upload failed: ") + cudaGetErrorString(e));
  }
  c->d_tables = d;
  c->dt = tables_at(c, d);
  return QF_OK;
}

struct Obs {
  uint32_t x = 0, z = 0, y = 0;
};

// Circuit qubit q to simulated bit (q + s) mod n, for a mask of qubits.
uint32_t rotate_mask(uint32_t m, int s, int n) {
  if (s == 0 || n <= 0) return m;
  const uint32_t all = n >= 32 ? ~0u : ((1u << n) - 1u);
  return ((m << s) | (m >> (n - s))) & all;
}

qf_status check_obs(const qf_circuit* c, qf_pauli obs, Obs* o) {
  const uint64_t valid = (c->circ.n >= 64) ? ~0ull : ((1ull << c->circ.n) - 1);
  if ((obs.x_mask | obs.z_mask) & ~valid)
    return fail(QF_ERR_INVALID_ARG, "observable acts on a qubit outside the circuit");
  o->y = (uint32_t)__builtin_popcountll(obs.x_mask & obs.z_mask) & 3u;
  // fused plans simulate the qubits in the plan's layout
  const int s = c->path == QF_PATH_FUSED ? c->fp.qshift : 0;
  o->x = rotate_mask((uint32_t)obs.x_mask, s, c->circ.n);
  o->z = rotate_mask((uint32_t)obs.z_mask, s, c->circ.n);
  return QF_OK;
}

qf_status check_precision(const qf_circuit* c, bool f64) {
  if (c->f64 == f64) return QF_OK;
  return fail(QF_ERR_INVALID_ARG, f64 ? "the plan is complex64: use the entry points without the 64 suffix"
                                      : "the plan is complex128 (QF_PREC_C128): use the *64 entry points");
}

qf_status check_call(const qf_circuit* c, int64_t batch, void* ws, size_t ws_bytes, bool f64 = false) {
  if (!c) return fail(QF_ERR_INVALID_ARG, "null circuit");
  if (!c->planned) return fail(QF_ERR_WORKSPACE, "circuit has no plan (call qf_plan)");
  if (check_precision(c, f64) != QF_OK) return QF_ERR_INVALID_ARG;
  if (c->host_only || !c->d_tables) return fail(QF_ERR_WORKSPACE, "plan was built host-only");
  if (batch < 0 || batch > c->batch) return fail(QF_ERR_INVALID_ARG, "batch exceeds the planned batch");
  if (!ws) return fail(QF_ERR_INVALID_ARG, "null workspace");
  if (((uintptr_t)ws & 255) != 0) return fail(QF_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < c->L.total) return fail(QF_ERR_WORKSPACE, "workspace smaller than qf_plan reported");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QF_ERR_CUDA, std::string("pending CUDA error: ") + cudaGetErrorString(e));
  return QF_OK;
}

#define QF_CU(call)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return fail(QF_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

// Run a train step through graph G: the first call with a key runs run(st)
// eagerly; the second records run on the handle's own stream and replays the
// graph on st; later calls with the key replay. A new key drops the graph. A
// step issued while st is being captured (by the caller) runs eagerly. With
// pass timing on (qf_profile), the graph holds the timing events of its
// passes in slots 0 .. ev_pairs-1: it is recorded and replayed only when no
// earlier timings are unread (qf_profile_read between steps), otherwise the
// step runs eagerly and appends its timings.
template <class F>
qf_status graph_step(qf_circuit* c, StepGraph& G, const std::array<uint64_t, 12>& key, cudaStream_t st, F&& run) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
      (c->profile && c->ev_used != 0)) {
    cudaGetLastError();
    return run(st);
  }
  if (G.key != key || G.profile != c->profile) {
    drop_graph(G);
    G.key = key;
    G.profile = c->profile;
  }
  if (!G.exec && G.seen && !G.failed) {
    if (!c->g_stream && cudaStreamCreateWithFlags(&c->g_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      c->g_stream = nullptr;
    }
    cudaGraph_t g = nullptr;
    G.failed = true;
    if (c->g_stream && cudaStreamBeginCapture(c->g_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      c->recording = true;
      const qf_status sc = run(c->g_stream);
      c->recording = false;
      const cudaError_t ec = cudaStreamEndCapture(c->g_stream, &g);
      if (sc == QF_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&G.exec, g, 0) == cudaSuccess) {
        G.launches = c->launches;
        G.failed = false;
        c->g_recorded++;
        G.ev_pairs = c->profile ? c->ev_used : 0;
        G.ev_dir.assign(c->ev_dir.begin(), c->ev_dir.begin() + G.ev_pairs);
        G.ev_launches.assign(c->ev_launches.begin(), c->ev_launches.begin() + G.ev_pairs);
      } else {
        G.exec = nullptr;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    c->ev_used = 0;  // the recording ran nothing
  }
  if (G.exec) {
    QF_CU(cudaGraphLaunch(G.exec, st));
    c->g_replayed++;
    c->launches = G.launches;
    if (c->profile) {
      std::copy(G.ev_dir.begin(), G.ev_dir.end(), c->ev_dir.begin());
      std::copy(G.ev_launches.begin(), G.ev_launches.end(), c->ev_launches.begin());
      c->ev_used = G.ev_pairs;
    }
    return QF_OK;
  }
  const qf_status s = run(st);
  if (s == QF_OK) G.seen = true;
  return s;
}

// x-mask in the tile coordinates of a pass; false when a bit is outside it.
bool local_xmask(const qf::PassDesc& pd, uint32_t xm, uint32_t* out) {
  uint32_t r = 0;
  for (int q = 0; q < 32; ++q) {
    if (!((xm >> q) & 1u)) continue;
    int lb = -1;
    for (int j = 0; j < pd.K; ++j)
      if (pd.gmap[j] == q) lb = j;
    if (lb < 0) return false;
    r |= 1u << lb;
  }
  *out = r;
  return true;
}

// Given initial states (QF_ENC_STATE_IN) are read by the pass that would
// generate psi_0.
void set_input(const qf_circuit* c, const float* x, qf::PassArgs& a) {
  a.psi_in = c->encoding == QF_ENC_STATE_IN ? reinterpret_cast<const float2*>(x) : nullptr;
  a.n_in = c->circ.n;
}

// The backward's parameter tables: (cos, sin) per gradient term for generic
// programs, the backward round parameters for round programs.
void set_term_table(const qf_circuit* c, const DevTables& T, const Layout& L, void* ws, qf::PrepArgs& pa) {
  pa.term_off = T.term_off;
  pa.term_params = T.term_params;
  pa.term_const = T.term_const;
  if (c->path == QF_PATH_FUSED && c->fp.rounds) {
    pa.n_terms = 0;
    pa.n_rpb = (int32_t)(c->fp.bwd_rounds.size() / qf::kBwdRoundWords);
    pa.rpb_src = T.bwd_rounds;
    pa.rpb_terms = T.bwd_rterms;
    pa.rpb = at<float4>(ws, L.rpb);
  } else {
    pa.n_terms = n_slots_of(c);
    pa.cs = at<float2>(ws, L.cs);
  }
}

// with_terms: also fill the backward's term table in the same prep launch
// (used by the train step, where the backward follows with the same theta).
// The loss of a train step, computed with the forward's E reduction when the
// batch allows one single-block launch for both (done is then set).
struct StepLoss {
  int32_t kind;
  const void* y;  // float32 labels (complex64 plans) or float64 (complex128 plans)
  double* loss;
  double* dLdE;
  bool done = false;
};

qf_status check_loss(int32_t kind, const double* E_d, const void* y_d, int64_t batch, const double* loss_d,
                     const double* dLdE_d) {
  if (kind != QF_LOSS_SUM && kind != QF_LOSS_MSE) return fail(QF_ERR_INVALID_ARG, "unknown loss");
  if (batch < 0 || (batch > 0 && (!E_d || !dLdE_d)) || !loss_d || (kind == QF_LOSS_MSE && batch > 0 && !y_d))
    return fail(QF_ERR_INVALID_ARG, "bad loss arguments");
  return QF_OK;
}

qf_status fused_forward(qf_circuit* c, const DevTables& T, const Layout& L, const float* theta, const float* x,
                        int64_t B, const Obs& o, double* E, void* ws, cudaStream_t st, bool with_terms = false,
                        StepLoss* sl = nullptr) {
  const qf::FusedPlan& P = c->fp;
  qf::PrepArgs pa{};
  pa.theta = theta;
  // round programs take their rotations and diagonals from the round tables;
  // the fused 2x2s are needed by generic steps and the tensor-core tables
  pa.n_fused = P.rounds && !c->tc ? 0 : (int32_t)P.fuse_off.size() - 1;
  pa.fuse_off = T.fuse_off;
  pa.fuse_gates = T.fuse_gates;
  pa.mats = at<float4>(ws, L.mats);
  pa.n_terms = 0;  // the forward needs the fused matrices, the encoding and the round parameters
  pa.term_off = T.term_off;  // round parameters are built from the gradient terms
  pa.term_params = T.term_params;
  pa.term_const = T.term_const;
  if (with_terms) set_term_table(c, T, L, ws, pa);
  if (P.rounds) {
    pa.n_rpf = (int32_t)(P.fwd_rounds.size() / qf::kFwdRoundWords);
    pa.rpf_src = T.fwd_rounds;
    pa.rpf_terms = T.fwd_rterms;
    pa.rpf = at<float4>(ws, L.rpf);
  }
  if (c->tc) pa.mats64 = at<double>(ws, L.mats64);
  pa.x = x;
  pa.B = c->encoding == QF_ENC_RY_X ? B : 0;  // given states need no encoding table
  pa.n = c->circ.n;
  pa.n_eff = P.n_eff;
  pa.qshift = P.qshift;
  pa.enc = at<float2>(ws, L.enc);
  // a train step's loss rides on the pass that computes the expectation (its
  // last CTA), or on the E-reduction launch
  const bool loss_in_pass = sl && B > 0 && qf::e_loss_fusable(B, (int)L.rows);
  if (loss_in_pass) pa.zero_word = at<uint32_t>(ws, L.done);
  QF_CU(qf::launch_prep(pa, st));
  c->call_launches++;
  if (c->tc) {
    QF_CU(qf::launch_tc_tables(T.fwd_rounds, (int32_t)(P.fwd_rounds.size() / qf::kFwdRoundWords), pa.mats64,
                               at<float>(ws, L.tcb), st));
    c->call_launches++;
  }
  qf::PassArgs a{};
  a.n_eff = P.n_eff;
  a.tps_log2 = P.n_eff - P.K;
  a.B = B;
  a.ops = T.fwd_ops;
  a.tcb = c->tc ? at<float>(ws, L.tcb) : nullptr;
  set_input(c, x, a);
  a.rounds = P.rounds ? T.fwd_rounds : nullptr;
  a.rx_items = P.has_rx ? 1 : 0;
  a.rpar = P.rounds ? at<float4>(ws, L.rpf) : nullptr;
  a.mats = pa.mats;
  a.cs = pa.cs;
  a.enc = pa.enc;
  a.work = at<float2>(ws, L.work);
  a.lam = at<float2>(ws, L.lam);
  a.slots = at<float2>(ws, L.slots);
  a.hslots = L.hslots ? at<char>(ws, L.hslots) : nullptr;
  a.slot_stride = L.state_elems;
  a.z_mask = o.z;
  a.y_count = o.y;
  a.e_part = at<double>(ws, L.epart);
  a.g_part = at<double>(ws, L.gpart);
  a.n_slots = P.n_terms;
  const int prof = prof_begin(c, st);
  int32_t full_expect = -1;  // slot of psi_M when the observable reaches outside the last tile
  bool loss_done = false;
  for (size_t pi = 0; pi < P.fwd.size(); ++pi) {
    a.pd = P.fwd[pi];
    a.pd.xm_local = 0;
    if ((a.pd.flags & qf::PF_EXPECT) && !local_xmask(a.pd, o.x, &a.pd.xm_local)) {
      a.pd.flags &= ~qf::PF_EXPECT;
      full_expect = a.pd.psi_dst;
    }
    a.done = nullptr;
    if (loss_in_pass && (a.pd.flags & qf::PF_EXPECT)) {
      a.done = at<uint32_t>(ws, L.done);
      a.E = E;
      a.y = static_cast<const float*>(sl->y);
      a.loss = sl->loss;
      a.dLdE_out = sl->dLdE;
      a.loss_kind = sl->kind;
      a.loss_scale = 2.0 / (double)B;
      loss_done = true;
    }
    if (c->tc) QF_CU(qf::launch_pass_tc(a, st));
    else QF_CU(qf::launch_pass(false, a, st, c->fwd_ctas));
    c->call_launches++;
  }
  prof_end(c, prof, 0, (int64_t)P.fwd.size(), st);
  if (full_expect >= 0) {
    QF_CU(qf::launch_expect_full(a.slots + (int64_t)full_expect * a.slot_stride, P.n_eff, B, L.rows, o.x, o.z,
                                 o.y, a.e_part, st));
    c->call_launches++;
  }
  if (loss_done) {
    sl->done = true;
  } else if (sl && qf::e_loss_fusable(B, (int)L.rows)) {
    QF_CU(qf::launch_e_loss(a.e_part, (int)L.rows, sl->kind, E, static_cast<const float*>(sl->y), B, sl->loss,
                            sl->dLdE, st));
    sl->done = true;
    c->call_launches++;
  } else {
    QF_CU(qf::launch_e_reduce(a.e_part, B, (int)L.rows, E, st));
    c->call_launches++;
  }
  return QF_OK;
}

// Observable reaching outside the seeding pass's tile: lambda_M for every
// amplitude as its own pass (psi_M from the pass's source slot).
cudaError_t seed_full(qf_circuit* c, const qf::FusedPlan& P, const qf::PassArgs& a, int64_t B, const Obs& o,
                      cudaStream_t st) {
  c->call_launches++;
  return qf::launch_seed_full(a.slots + (int64_t)a.pd.psi_src * a.slot_stride, a.lam, P.n_eff, B, o.x, o.z, o.y,
                              a.dLdE, st);
}

// with_prep = false: the term table was filled by the preceding forward.
qf_status fused_backward(qf_circuit* c, const DevTables& T, const Layout& L, const float* theta, const float* x,
                         int64_t B, const Obs& o, const double* dLdE, double* grad, int per_sample, void* ws,
                         cudaStream_t st, bool with_prep = true) {
  const qf::FusedPlan& P = c->fp;
  qf::PrepArgs pa{};
  pa.theta = theta;
  pa.n_fused = 0;
  set_term_table(c, T, L, ws, pa);
  pa.B = 0;
  pa.n = c->circ.n;
  pa.n_eff = P.n_eff;
  if (with_prep) {
    QF_CU(qf::launch_prep(pa, st));
    c->call_launches++;
  }
  qf::PassArgs a{};
  a.n_eff = P.n_eff;
  a.tps_log2 = P.n_eff - P.K;
  a.B = B;
  a.ops = T.bwd_ops;
  a.rounds = P.rounds ? T.bwd_rounds : nullptr;
  a.rx_items = P.has_rx ? 1 : 0;
  a.rpar = P.rounds ? at<float4>(ws, L.rpb) : nullptr;
  a.cs = pa.cs;
  a.work = at<float2>(ws, L.work);
  a.lam = at<float2>(ws, L.lam);
  a.slots = at<float2>(ws, L.slots);
  a.hslots = L.hslots ? at<char>(ws, L.hslots) : nullptr;
  a.slot_stride = L.state_elems;
  a.z_mask = o.z;
  a.y_count = o.y;
  a.dLdE = dLdE;
  a.e_part = at<double>(ws, L.epart);
  a.g_part = at<double>(ws, L.gpart);
  a.n_slots = P.n_terms;
  const int prof = prof_begin(c, st);
  if (P.ckpt_mode == 1) {
    // checkpoint mode A: forward re-runs (tables and encodings of the preceding
    // forward) interleaved with adjoint passes, block by block
    qf::PassArgs f = a;
    f.ops = T.fwd_ops;
    f.rounds = P.rounds ? T.fwd_rounds : nullptr;
    f.rpar = P.rounds ? at<float4>(ws, L.rpf) : nullptr;
    f.mats = at<float4>(ws, L.mats);
    f.enc = at<float2>(ws, L.enc);
    f.tcb = c->tc ? at<float>(ws, L.tcb) : nullptr;
    set_input(c, x, f);
    for (size_t i = 0; i < P.a_sched.size(); ++i) {
      const bool bwd = P.a_dir[i] != 0;
      qf::PassArgs& x = bwd ? a : f;
      x.pd = P.a_sched[i];
      x.pd.xm_local = 0;
      if (bwd && x.pd.lam_src == qf::LAM_SEED && !local_xmask(x.pd, o.x, &x.pd.xm_local)) {
        QF_CU(seed_full(c, P, x, B, o, st));
        x.pd.lam_src = qf::LAM_BUF;
      }
      if (c->tc && !bwd) QF_CU(qf::launch_pass_tc(x, st));
      else QF_CU(qf::launch_pass(bwd, x, st, c->fwd_ctas));
      c->call_launches++;
    }
    prof_end(c, prof, 1, (int64_t)P.a_sched.size(), st);
  } else {
    for (size_t pi = 0; pi < P.bwd.size(); ++pi) {
      a.pd = P.bwd[pi];
      a.pd.xm_local = 0;
      if (a.pd.lam_src == qf::LAM_SEED && !local_xmask(a.pd, o.x, &a.pd.xm_local)) {
        QF_CU(seed_full(c, P, a, B, o, st));
        a.pd.lam_src = qf::LAM_BUF;
      }
      QF_CU(qf::launch_pass(true, a, st));
      c->call_launches++;
    }
    prof_end(c, prof, 1, (int64_t)P.bwd.size(), st);
  }
  qf::GradReduceArgs g{};
  g.g_part = a.g_part;
  g.B = B;
  g.tps = L.rows;
  g.slot_stride = P.n_terms;
  g.slot_step = 1;
  g.n_params = c->circ.n_params;
  g.param_off = T.param_off;
  g.param_slots = T.param_terms;
  g.per_sample = per_sample;
  g.grad = grad;
  g.scratch = L.gred ? at<double>(ws, L.gred) : nullptr;
  QF_CU(qf::launch_g_reduce(g, st));
  c->call_launches += qf::g_reduce_stages(g.tps, g.slot_step);
  return QF_OK;
}

// ---- complex128 plans: the same pass sequences on the float64 kernels ----------
qf::PassArgs64 pass_args64(const qf_circuit* c, const Layout& L, void* ws, int64_t B, const Obs& o) {
  const qf::FusedPlan& P = c->fp;
  qf::PassArgs64 a{};
  a.n_eff = P.n_eff;
  a.tps_log2 = P.n_eff - P.K;
  a.B = B;
  a.mats = at<double2>(ws, L.mats64);
  a.cs = at<double2>(ws, L.cs);
  a.rounds = nullptr;
  a.rpar = nullptr;
  a.rx_items = P.has_rx ? 1 : 0;
  a.enc = at<double2>(ws, L.enc);
  a.n_in = c->circ.n;
  a.work = at<double2>(ws, L.work);
  a.lam = at<double2>(ws, L.lam);
  a.slots = at<double2>(ws, L.slots);
  a.fslots = L.hslots ? at<float2>(ws, L.hslots) : nullptr;
  a.slot_stride = L.state_elems;
  a.z_mask = o.z;
  a.y_count = o.y;
  a.e_part = at<double>(ws, L.epart);
  a.g_part = at<double>(ws, L.gpart);
  a.n_slots = P.n_terms;
  return a;
}

// Prep arguments of a complex128 plan: fused 2x2s, terms and encodings in float64.
qf::PrepArgs prep_args64(const qf_circuit* c, const DevTables& T, const Layout& L, void* ws, const double* theta) {
  qf::PrepArgs pa{};
  pa.theta64 = theta;
  pa.fuse_off = T.fuse_off;
  pa.fuse_gates = T.fuse_gates;
  pa.mats64 = at<double>(ws, L.mats64);
  pa.term_off = T.term_off;
  pa.term_params = T.term_params;
  pa.term_const = T.term_const;
  pa.cs64 = at<double2>(ws, L.cs);
  pa.n = c->circ.n;
  pa.n_eff = c->fp.n_eff;
  pa.qshift = c->fp.qshift;
  pa.enc64 = at<double2>(ws, L.enc);
  return pa;
}

// The backward round parameters of a complex128 round program.
void set_rounds64(const qf_circuit* c, const DevTables& T, const Layout& L, void* ws, qf::PrepArgs& pa) {
  pa.n_rpb = (int32_t)(c->fp.bwd_rounds.size() / qf::kBwdRoundWords);
  pa.rpb_src = T.bwd_rounds;
    pa.rpb_terms = T.bwd_rterms;
  pa.rpb64 = at<qf::RoundPar64>(ws, L.rpb);
}

qf_status fused_forward64(qf_circuit* c, const DevTables& T, const Layout& L, const double* theta, const double* x,
                          int64_t B, const Obs& o, double* E, void* ws, cudaStream_t st, bool with_terms = false,
                          StepLoss* sl = nullptr) {
  const qf::FusedPlan& P = c->fp;
  qf::PrepArgs pa = prep_args64(c, T, L, ws, theta);
  if (P.rounds) {
    // round programs: the forward's and (with_terms) the backward's round parameters
    pa.n_fused = 0;
    pa.n_rpf = (int32_t)(P.fwd_rounds.size() / qf::kFwdRoundWords);
    pa.rpf_src = T.fwd_rounds;
    pa.rpf_terms = T.fwd_rterms;
    pa.rpf64 = at<qf::RoundPar64>(ws, L.rpf);
    if (with_terms) set_rounds64(c, T, L, ws, pa);
  } else {
    pa.n_fused = (int32_t)P.fuse_off.size() - 1;
    pa.n_terms = with_terms ? P.n_terms : 0;
  }
  pa.x64 = x;
  pa.B = c->encoding == QF_ENC_RY_X ? B : 0;
  QF_CU(qf::launch_prep(pa, st));
  c->call_launches++;
  qf::PassArgs64 a = pass_args64(c, L, ws, B, o);
  a.ops = T.fwd_ops;
  if (P.rounds) {
    a.rounds = T.fwd_rounds;
    a.rpar = at<qf::RoundPar64>(ws, L.rpf);
  }
  a.psi_in = c->encoding == QF_ENC_STATE_IN ? reinterpret_cast<const double2*>(x) : nullptr;
  const int prof = prof_begin(c, st);
  int32_t full_expect = -1;
  for (size_t pi = 0; pi < P.fwd.size(); ++pi) {
    a.pd = P.fwd[pi];
    a.pd.xm_local = 0;
    if ((a.pd.flags & qf::PF_EXPECT) && !local_xmask(a.pd, o.x, &a.pd.xm_local)) {
      a.pd.flags &= ~qf::PF_EXPECT;
      full_expect = a.pd.psi_dst;
    }
    QF_CU(qf::launch_pass64(false, a, st));
    c->call_launches++;
  }
  prof_end(c, prof, 0, (int64_t)P.fwd.size(), st);
  if (full_expect >= 0) {
    QF_CU(qf::launch_expect_full64(a.slots + (int64_t)full_expect * a.slot_stride, P.n_eff, B, L.rows, o.x, o.z,
                                   o.y, a.e_part, st));
    c->call_launches++;
  }
  if (sl && qf::e_loss_fusable(B, (int)L.rows)) {
    QF_CU(qf::launch_e_loss64(a.e_part, (int)L.rows, sl->kind, E, static_cast<const double*>(sl->y), B, sl->loss,
                              sl->dLdE, st));
    sl->done = true;
  } else {
    QF_CU(qf::launch_e_reduce(a.e_part, B, (int)L.rows, E, st));
  }
  c->call_launches++;
  return QF_OK;
}

qf_status fused_backward64(qf_circuit* c, const DevTables& T, const Layout& L, const double* theta,
                           const double* x, int64_t B, const Obs& o, const double* dLdE, double* grad,
                           int per_sample, void* ws, cudaStream_t st, bool with_prep = true) {
  const qf::FusedPlan& P = c->fp;
  if (with_prep) {
    qf::PrepArgs pa = prep_args64(c, T, L, ws, theta);
    if (P.rounds) set_rounds64(c, T, L, ws, pa);
    else pa.n_terms = P.n_terms;
    QF_CU(qf::launch_prep(pa, st));
    c->call_launches++;
  }
  qf::PassArgs64 a = pass_args64(c, L, ws, B, o);
  a.ops = T.bwd_ops;
  a.dLdE = dLdE;
  if (P.rounds) {
    a.rounds = T.bwd_rounds;
    a.rpar = at<qf::RoundPar64>(ws, L.rpb);
  }
  auto seed = [&](const qf::PassArgs64& p) -> cudaError_t {
    c->call_launches++;
    return qf::launch_seed_full64(p.slots + (int64_t)p.pd.psi_src * p.slot_stride, p.lam, P.n_eff, B, o.x, o.z,
                                  o.y, p.dLdE, st);
  };
  const int prof = prof_begin(c, st);
  if (P.ckpt_mode == 1) {
    // checkpoint mode A: forward re-runs interleaved with adjoint passes
    qf::PassArgs64 f = a;
    f.ops = T.fwd_ops;
    if (P.rounds) {
      f.rounds = T.fwd_rounds;
      f.rpar = at<qf::RoundPar64>(ws, L.rpf);
    }
    f.psi_in = c->encoding == QF_ENC_STATE_IN ? reinterpret_cast<const double2*>(x) : nullptr;
    for (size_t i = 0; i < P.a_sched.size(); ++i) {
      const bool bwd = P.a_dir[i] != 0;
      qf::PassArgs64& p = bwd ? a : f;
      p.pd = P.a_sched[i];
      p.pd.xm_local = 0;
      if (bwd && p.pd.lam_src == qf::LAM_SEED && !local_xmask(p.pd, o.x, &p.pd.xm_local)) {
        QF_CU(seed(p));
        p.pd.lam_src = qf::LAM_BUF;
      }
      QF_CU(qf::launch_pass64(bwd, p, st));
      c->call_launches++;
    }
    prof_end(c, prof, 1, (int64_t)P.a_sched.size(), st);
  } else {
    for (size_t pi = 0; pi < P.bwd.size(); ++pi) {
      a.pd = P.bwd[pi];
      a.pd.xm_local = 0;
      if (a.pd.lam_src == qf::LAM_SEED && !local_xmask(a.pd, o.x, &a.pd.xm_local)) {
        QF_CU(seed(a));
        a.pd.lam_src = qf::LAM_BUF;
      }
      QF_CU(qf::launch_pass64(true, a, st));
      c->call_launches++;
    }
    prof_end(c, prof, 1, (int64_t)P.bwd.size(), st);
  }
  qf::GradReduceArgs g{};
  g.g_part = a.g_part;
  g.B = B;
  g.tps = L.rows;
  g.slot_stride = P.n_terms;
  g.slot_step = 1;
  g.n_params = c->circ.n_params;
  g.param_off = T.param_off;
  g.param_slots = T.param_terms;
  g.per_sample = per_sample;
  g.grad = grad;
  g.scratch = L.gred ? at<double>(ws, L.gred) : nullptr;
  QF_CU(qf::launch_g_reduce(g, st));
  c->call_launches += qf::g_reduce_stages(g.tps, g.slot_step);
  return QF_OK;
}

qf_status pg_forward(qf_circuit* c, const DevTables& T, const Layout& L, const float* theta, const float* x,
                     int64_t B, const Obs& o, double* E, void* ws, cudaStream_t st) {
  const qf::PerGatePlan& P = c->gp;
  qf::PrepArgs pa{};
  pa.theta = theta;
  pa.n_terms = n_slots_of(c);
  pa.term_off = T.term_off;
  pa.term_params = T.term_params;
  pa.term_const = T.term_const;
  pa.cs = at<float2>(ws, L.cs);
  pa.x = x;
  pa.B = c->encoding == QF_ENC_RY_X ? B : 0;
  pa.n = c->circ.n;
  pa.n_eff = P.n_eff;
  pa.enc = at<float2>(ws, L.enc);
  QF_CU(qf::launch_prep(pa, st));
  c->call_launches++;
  qf::PerGateArgs a{P.n_eff, B, at<float2>(ws, L.work), at<float2>(ws, L.lam), (int32_t)L.rows};
  if (B == 0) return QF_OK;
  if (c->encoding == QF_ENC_STATE_IN) QF_CU(qf::pg_load_states(a, reinterpret_cast<const float2*>(x), c->circ.n, st));
  else QF_CU(qf::pg_encode(a, pa.enc, st));
  c->call_launches++;
  size_t k = 0;
  int slot = 0;
  for (int g = 0; g < (int)c->circ.gates.size(); ++g) {
    const qf::Gate& gt = c->circ.gates[g];
    if (gt.kind == qf::G_CZ) {
      QF_CU(qf::pg_cz(a, gt.q0, gt.q1, false, st));
    } else if (gt.kind == qf::G_CNOT) {
      QF_CU(qf::pg_cnot(a, gt.q0, gt.q1, false, st));
    } else {
      QF_CU(qf::pg_rot(a, gt.kind, gt.q0, pa.cs, slot++, st));
    }
    c->call_launches++;
    if (k < P.ckpt_after.size() && P.ckpt_after[k] == g) {
      QF_CU(qf::pg_copy(a.psi, at<float2>(ws, L.slots) + (int64_t)k * L.state_elems, L.state_elems, st));
      c->call_launches++;
      ++k;
    }
  }
  QF_CU(qf::pg_expect(a, o.x, o.z, o.y, at<double>(ws, L.epart), st));
  QF_CU(qf::launch_e_reduce(at<double>(ws, L.epart), B, (int)L.rows, E, st));
  c->call_launches += 2;
  return QF_OK;
}

qf_status pg_backward(qf_circuit* c, const DevTables& T, const Layout& L, const float* theta, int64_t B,
                      const Obs& o, const double* dLdE, double* grad, int per_sample, void* ws, cudaStream_t st) {
  const qf::PerGatePlan& P = c->gp;
  qf::PrepArgs pa{};
  pa.theta = theta;
  pa.n_terms = n_slots_of(c);
  pa.term_off = T.term_off;
  pa.term_params = T.term_params;
  pa.term_const = T.term_const;
  pa.cs = at<float2>(ws, L.cs);
  pa.n = c->circ.n;
  pa.n_eff = P.n_eff;
  QF_CU(qf::launch_prep(pa, st));
  c->call_launches++;
  qf::PerGateArgs a{P.n_eff, B, at<float2>(ws, L.work), at<float2>(ws, L.lam), (int32_t)L.rows};
  double* gpart = at<double>(ws, L.gpart);
  if (B > 0) {
    QF_CU(qf::pg_seed(a, o.x, o.z, o.y, dLdE, st));
    c->call_launches++;
    int k = (int)P.ckpt_after.size() - 1;
    int slot = P.n_slots - 1;
    for (int g = (int)c->circ.gates.size() - 1; g >= 0; --g) {
      if (k >= 0 && P.ckpt_after[k] == g) {
        // re-anchor psi to the stored state after gate g
        QF_CU(qf::pg_copy(at<float2>(ws, L.slots) + (int64_t)k * L.state_elems, a.psi, L.state_elems, st));
        c->call_launches++;
        --k;
      }
      const qf::Gate& gt = c->circ.gates[g];
      if (gt.kind == qf::G_CZ) {
        QF_CU(qf::pg_cz(a, gt.q0, gt.q1, true, st));
      } else if (gt.kind == qf::G_CNOT) {
        QF_CU(qf::pg_cnot(a, gt.q0, gt.q1, true, st));
      } else {
        QF_CU(qf::pg_rot_bwd(a, gt.kind, gt.q0, pa.cs, slot, gpart + (int64_t)slot * B * L.rows, st));
        --slot;
      }
      c->call_launches++;
    }
  }
  qf::GradReduceArgs g{};
  g.g_part = gpart;
  g.B = B;
  g.tps = L.rows;
  g.slot_stride = 1;
  g.slot_step = B * L.rows;
  g.n_params = c->circ.n_params;
  g.param_off = T.param_off;
  g.param_slots = T.param_terms;
  g.per_sample = per_sample;
  g.grad = grad;
  g.scratch = L.gred ? at<double>(ws, L.gred) : nullptr;
  QF_CU(qf::launch_g_reduce(g, st));
  c->call_launches += qf::g_reduce_stages(g.tps, g.slot_step);
  return QF_OK;
}

}  // namespace

extern "C" {

qf_status qf_check_bounded_wait(void* stream, int64_t spin_limit) {
  if (spin_limit < 1 || spin_limit > (1 << 20)) return fail(QF_ERR_INVALID_ARG, "spin_limit must be in 1..2^20");
  QF_CU(qf::bounded_wait_probe((long long)spin_limit, static_cast<cudaStream_t>(stream)));
  return QF_OK;
}

qf_status qf_device_status(void* stream, int32_t* code) {
  if (!code) return fail(QF_ERR_INVALID_ARG, "null argument");
  *code = 0;
  QF_CU(qf::device_status(code, static_cast<cudaStream_t>(stream)));
  return QF_OK;
}

const char* qf_last_error(void) { return g_err.c_str(); }

int32_t qf_version(void) { return 100; }

qf_status qf_hea_create(int32_t n_qubits, int32_t n_layers, int32_t entangler, int32_t encoding,
                        qf_circuit** out) {
  if (!out) return fail(QF_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (encoding != QF_ENC_RY_X && encoding != QF_ENC_STATE_IN) return fail(QF_ERR_INVALID_ARG, "unknown encoding");
  try {
    qf_circuit* c = new qf_circuit();
    c->encoding = encoding;
    try {
      qf::build_hea(c->circ, n_qubits, n_layers, entangler);
    } catch (...) {
      delete c;
      throw;
    }
    *out = c;
    return QF_OK;
  } catch (const std::bad_alloc&) {
    return fail(QF_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(QF_ERR_INVALID_ARG, e.what());
  }
}

qf_status qf_circuit_create(int32_t n_qubits, const qf_gate* gates, int32_t n_gates, int32_t n_params,
                            int32_t encoding, qf_circuit** out) {
  if (!out) return fail(QF_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (n_gates < 0 || (n_gates > 0 && !gates)) return fail(QF_ERR_INVALID_ARG, "bad gate array");
  if (encoding != QF_ENC_RY_X && encoding != QF_ENC_STATE_IN) return fail(QF_ERR_INVALID_ARG, "unknown encoding");
  try {
    qf_circuit* c = new qf_circuit();
    c->encoding = encoding;
    c->circ.n = n_qubits;
    c->circ.n_params = n_params;
    for (int i = 0; i < n_gates; ++i) {
      qf::Gate g{gates[i].kind, gates[i].q0, gates[i].q1, gates[i].param};
      if (g.kind == qf::G_CZ || g.kind == qf::G_CNOT) g.param = -1;
      else g.q1 = -1;
      c->circ.gates.push_back(g);
    }
    try {
      qf::validate_circuit(c->circ);
    } catch (...) {
      delete c;
      throw;
    }
    *out = c;
    return QF_OK;
  } catch (const std::bad_alloc&) {
    return fail(QF_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(QF_ERR_INVALID_ARG, e.what());
  }
}

qf_status qf_circuit_destroy(qf_circuit* c) {
  if (!c) return QF_OK;
  free_tables(c);     // drops the step graphs, which may hold the timing events
  destroy_events(c);
  if (c->g_stream) cudaStreamDestroy(c->g_stream);
  delete c;
  return QF_OK;
}

qf_status qf_plan(qf_circuit* c, const qf_plan_opts* opts, int64_t batch, size_t* workspace_bytes) {
  if (!c) return fail(QF_ERR_INVALID_ARG, "null circuit");
  if (batch < 0) return fail(QF_ERR_INVALID_ARG, "negative batch");
  qf_plan_opts o{};
  if (opts) o = *opts;
  if (o.path != QF_PATH_FUSED && o.path != QF_PATH_PER_GATE) return fail(QF_ERR_INVALID_ARG, "unknown path");
  if (o.tile_bits != 0 && (o.tile_bits < 4 || o.tile_bits > 12))
    return fail(QF_ERR_INVALID_ARG, "tile_bits must be 0 or in 4..12");
  if (o.ckpt_layers < 0) return fail(QF_ERR_INVALID_ARG, "negative checkpoint interval");
  if (o.program != 0 && o.program != 1) return fail(QF_ERR_INVALID_ARG, "program must be 0 or 1");
  if (o.ckpt_mode != 0 && o.ckpt_mode != 1) return fail(QF_ERR_INVALID_ARG, "ckpt_mode must be 0 or 1");
  if (o.mem_save != 0 && o.mem_save != 1) return fail(QF_ERR_INVALID_ARG, "mem_save must be 0 or 1");
  if (o.mem_save && o.ckpt_mode != 1) return fail(QF_ERR_INVALID_ARG, "mem_save needs ckpt_mode 1");
  if (o.ckpt_mode != 0 && o.path != QF_PATH_FUSED)
    return fail(QF_ERR_UNSUPPORTED, "ckpt_mode 1 applies to the fused path");
  if (o.tc_path != 0 && o.tc_path != 1) return fail(QF_ERR_INVALID_ARG, "tc_path must be 0 or 1");
  if (o.tc_path && o.path != QF_PATH_FUSED) return fail(QF_ERR_UNSUPPORTED, "tc_path applies to the fused path");
  if (o.precision != QF_PREC_C64 && o.precision != QF_PREC_C128)
    return fail(QF_ERR_INVALID_ARG, "precision must be QF_PREC_C64 or QF_PREC_C128");
  if (o.precision == QF_PREC_C128 && o.path != QF_PATH_FUSED)
    return fail(QF_ERR_UNSUPPORTED, "complex128 runs on the fused path");
  if (o.precision == QF_PREC_C128 && o.tc_path)
    return fail(QF_ERR_UNSUPPORTED, "the tensor-core path is complex64 (3xTF32)");
  if (o.catch_up < 0 || o.catch_up > 2) return fail(QF_ERR_INVALID_ARG, "catch_up must be 0, 1 or 2");
  if (o.fwd_ctas != 0 && o.fwd_ctas != 2 && o.fwd_ctas != 3)
    return fail(QF_ERR_INVALID_ARG, "fwd_ctas must be 0, 2 or 3");
  try {
    free_tables(c);
    c->planned = false;
    c->path = o.path;
    c->ckpt_layers = o.ckpt_layers > 0 ? o.ckpt_layers : 10;
    c->host_only = o.host_only != 0;
    c->staging = o.no_host_staging == 0;
    c->f64 = o.precision == QF_PREC_C128;
    c->batch = batch;
    qf::PlanRequest req;
    req.tile_bits = o.tile_bits;
    req.ckpt_layers = c->ckpt_layers;
    req.generic = o.program == 1;
    req.ckpt_mode = o.ckpt_mode;
    req.mem_save = o.mem_save != 0;
    // given states arrive in circuit order: their plans keep the identity layout
    req.relabel = c->encoding == QF_ENC_RY_X;
    req.catch_up = o.catch_up == 1 ? 1 : o.catch_up == 2 ? 0 : -1;
    c->fwd_ctas = o.fwd_ctas;
    if (c->lay_valid && c->lay_tile_bits == o.tile_bits && c->lay_generic == (int)req.generic &&
        c->lay_catch_up == o.catch_up) {
      req.qshift = c->lay_shift;
      req.strict = c->lay_strict;
    }
    c->tc = false;
    if (c->path == QF_PATH_FUSED) {
      c->fp = qf::plan_fused(c->circ, req);
      c->lay_valid = true;
      c->lay_tile_bits = o.tile_bits;
      c->lay_generic = (int)req.generic;
      c->lay_catch_up = o.catch_up;
      c->lay_shift = c->fp.qshift;
      c->lay_strict = c->fp.strict;
      c->gp = qf::PerGatePlan();
      if (o.tc_path) {
        if (!c->fp.rounds || c->fp.K != qf::kMaxTileBits)
          throw std::domain_error("tc_path needs round programs with 12-qubit tiles (n >= 12, RZ/RY, chain CZs)");
        c->tc = true;
      }
    } else {
      c->gp = qf::plan_per_gate(c->circ, req);
      c->fp = qf::FusedPlan();
    }
    c->L = make_layout(c, batch);
    build_blob(c);
  } catch (const std::domain_error& e) {
    return fail(QF_ERR_UNSUPPORTED, e.what());
  } catch (const std::bad_alloc&) {
    return fail(QF_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(QF_ERR_INVALID_ARG, e.what());
  }
  if (!c->host_only) {
    qf_status s = upload(c);
    if (s != QF_OK) return s;
  }
  c->planned = true;
  if (workspace_bytes) *workspace_bytes = c->L.total;
  return QF_OK;
}

double qf_mem_model(double k, double d, double b, double* b_best) {
  if (b_best) *b_best = (k > 0 && d > 0) ? std::sqrt(d / k) : 0.0;
  if (b <= 0) return 0.0;
  return k * b + d / b;
}

qf_status qf_plan_fit(qf_circuit* c, const qf_plan_opts* opts, int64_t batch, size_t mem_bytes, int32_t* ckpt_layers,
                      size_t* workspace_bytes) {
  if (!c || !ckpt_layers) return fail(QF_ERR_INVALID_ARG, "null argument");
  *ckpt_layers = 0;
  qf_plan_opts o{};
  if (opts) o = *opts;
  const int d = c->circ.layers > 0 ? c->circ.layers : std::max(1, (int)c->circ.gates.size());
  // the workspace shrinks as the interval grows: binary search on a host-only plan
  auto ws_for = [&](int cl, size_t* ws) -> qf_status {
    qf_plan_opts t = o;
    t.ckpt_layers = cl;
    t.host_only = 1;
    return qf_plan(c, &t, batch, ws);
  };
  size_t ws = 0;
  qf_status s;
  if (o.ckpt_mode == 1) {
    // mode A: the workspace is about (p c + d / c) states, smallest near
    // c = sqrt(d / p) (Eq. 8); its recompute costs about one forward for any
    // c. Take the c with the smallest workspace (ternary search on the
    // unimodal count, then a local scan) and fail if even that does not fit.
    std::map<int, size_t> memo;
    auto wsc = [&](int cl) -> size_t {
      auto it = memo.find(cl);
      if (it != memo.end()) return it->second;
      size_t w = 0;
      if (ws_for(cl, &w) != QF_OK) w = SIZE_MAX;
      memo[cl] = w;
      return w;
    };
    int lo = 1, hi = d;
    while (hi - lo > 4) {
      const int m1 = lo + (hi - lo) / 3, m2 = hi - (hi - lo) / 3;
      if (wsc(m1) <= wsc(m2)) hi = m2;
      else lo = m1;
    }
    int best = lo;
    for (int cl = lo; cl <= hi; ++cl)
      if (wsc(cl) < wsc(best)) best = cl;
    if (wsc(best) == SIZE_MAX) return fail(QF_ERR_INVALID_ARG, "planning failed");
    if (wsc(best) > mem_bytes) return fail(QF_ERR_WORKSPACE, "no checkpoint interval fits");
    qf_plan_opts fin = o;
    fin.ckpt_layers = best;
    if ((s = qf_plan(c, &fin, batch, &ws)) != QF_OK) return s;
    *ckpt_layers = best;
    if (workspace_bytes) *workspace_bytes = ws;
    return QF_OK;
  }
  s = ws_for(d, &ws);
  if (s != QF_OK) return s;
  if (ws > mem_bytes) return fail(QF_ERR_WORKSPACE, "even a plan with only the final state does not fit");
  int lo = 1, hi = d;  // hi fits
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if ((s = ws_for(mid, &ws)) != QF_OK) return s;
    if (ws <= mem_bytes) hi = mid;
    else lo = mid + 1;
  }
  qf_plan_opts fin = o;
  fin.ckpt_layers = hi;
  if ((s = qf_plan(c, &fin, batch, &ws)) != QF_OK) return s;
  *ckpt_layers = hi;
  if (workspace_bytes) *workspace_bytes = ws;
  return QF_OK;
}

qf_status qf_plan_info(const qf_circuit* c, qf_plan_info_t* info) {
  if (!c || !info) return fail(QF_ERR_INVALID_ARG, "null argument");
  if (!c->planned) return fail(QF_ERR_WORKSPACE, "circuit has no plan");
  memset(info, 0, sizeof(*info));
  info->n_qubits = c->circ.n;
  info->n_params = c->circ.n_params;
  info->path = c->path;
  info->ckpt_layers = c->ckpt_layers;
  info->batch = c->batch;
  info->workspace_bytes = (int64_t)c->L.total;
  info->state_bytes = c->L.state_elems * (c->f64 ? 16 : 8);
  info->precision = c->f64 ? QF_PREC_C128 : QF_PREC_C64;
  if (c->path == QF_PATH_FUSED) {
    info->n_eff = c->fp.n_eff;
    info->n_slots = c->fp.n_terms;
    info->tile_bits = c->fp.K;
    info->n_passes = (int32_t)c->fp.fwd.size();
    info->n_steps = c->fp.n_steps;
    info->n_fused_ops = (int32_t)c->fp.fuse_off.size() - 1;
    info->n_ckpt = c->fp.n_ckpt;
    info->launches_fwd = info->n_passes + 2;
    // a two-stage gradient reduction when a sample has many tile rows
    info->launches_bwd = info->n_passes + 1 + qf::g_reduce_stages(c->L.rows, 1);
    info->ckpt_mode = c->fp.ckpt_mode;
    info->mem_save = c->fp.mem_save ? 1 : 0;
    info->n_pass_slots = c->fp.n_aslots;
    info->tc_path = c->tc ? 1 : 0;
    info->qubit_shift = c->fp.qshift;
    info->catch_up = c->fp.rounds && c->fp.n_eff > c->fp.K ? (c->fp.strict ? 1 : 2) : 0;
    info->fwd_ctas = c->fwd_ctas;
    if (c->tc) info->launches_fwd += 1;  // the B-block table
    if (c->fp.ckpt_mode == 1) info->launches_bwd = (int32_t)c->fp.a_sched.size() + 1 + qf::g_reduce_stages(c->L.rows, 1);
  } else {
    info->n_eff = c->gp.n_eff;
    info->n_slots = c->gp.n_slots;
    info->n_passes = (int32_t)c->circ.gates.size();
    info->n_ckpt = c->gp.n_ckpt;
    const int M = (int)c->circ.gates.size(), k = (int)c->gp.ckpt_after.size();
    info->launches_fwd = M + k + 4;
    info->launches_bwd = M + k + 3;
  }
  return QF_OK;
}

}  // extern "C"

namespace {

// The argument key of a device-buffer train step.
std::array<uint64_t, 12> step_key(const void* theta, const void* x, const void* y, int64_t batch, int32_t loss_kind,
                                  qf_pauli obs, const void* loss, const void* E, const void* grad, const void* ws,
                                  size_t ws_bytes) {
  auto u = [](const void* p) { return (uint64_t)(uintptr_t)p; };
  return {u(theta), u(x), u(y), (uint64_t)batch, (uint64_t)loss_kind, obs.x_mask, obs.z_mask, u(loss), u(E), u(grad),
          u(ws), (uint64_t)ws_bytes};
}

qf_status train_step_eager(qf_circuit* c, const float* theta_d, const float* x_d, const float* y_d, int64_t batch,
                           int32_t loss_kind, qf_pauli obs, double* loss_d, double* E_d, double* grad_d, void* ws_d,
                           size_t ws_bytes, void* stream) {
  if (c && c->planned && c->path == QF_PATH_FUSED) {
    // fused: one prep launch fills the forward's and the backward's tables
    qf_status s = check_call(c, batch, ws_d, ws_bytes);
    if (s != QF_OK) return s;
    if ((!theta_d && c->circ.n_params > 0) || (batch > 0 && (!x_d || !E_d)) || !loss_d ||
        (!grad_d && c->circ.n_params > 0))
      return fail(QF_ERR_INVALID_ARG, "null data pointer");
    Obs o;
    if ((s = check_obs(c, obs, &o)) != QF_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* dLdE = at<double>(ws_d, c->L.dLdE);
    if ((s = check_loss(loss_kind, E_d, y_d, batch, loss_d, dLdE)) != QF_OK) return s;
    c->call_launches = 0;
    StepLoss sl{loss_kind, y_d, loss_d, dLdE};
    s = fused_forward(c, c->dt, c->L, theta_d, x_d, batch, o, E_d, ws_d, st, true, &sl);
    if (s != QF_OK) return s;
    if (!sl.done) {
      s = qf_loss(loss_kind, E_d, y_d, batch, loss_d, dLdE, stream);
      if (s != QF_OK) return s;
      c->call_launches++;
    }
    s = fused_backward(c, c->dt, c->L, theta_d, x_d, batch, o, dLdE, grad_d, 0, ws_d, st, false);
    c->launches = c->call_launches;
    return s;
  }
  qf_status s = qf_forward(c, theta_d, x_d, batch, obs, E_d, ws_d, ws_bytes, stream);
  if (s != QF_OK) return s;
  double* dLdE = at<double>(ws_d, c->L.dLdE);
  s = qf_loss(loss_kind, E_d, y_d, batch, loss_d, dLdE, stream);
  if (s != QF_OK) return s;
  const int64_t fwd_launches = c->launches;
  s = qf_backward(c, theta_d, x_d, batch, obs, dLdE, grad_d, 0, ws_d, ws_bytes, stream);
  c->launches = fwd_launches + 1 + c->call_launches;
  return s;
}

qf_status train_step_eager64(qf_circuit* c, const double* theta_d, const double* x_d, const double* y_d,
                             int64_t batch, int32_t loss_kind, qf_pauli obs, double* loss_d, double* E_d,
                             double* grad_d, void* ws_d, size_t ws_bytes, void* stream) {
  qf_status s = check_call(c, batch, ws_d, ws_bytes, true);
  if (s != QF_OK) return s;
  if ((!theta_d && c->circ.n_params > 0) || (batch > 0 && (!x_d || !E_d)) || !loss_d ||
      (!grad_d && c->circ.n_params > 0))
    return fail(QF_ERR_INVALID_ARG, "null data pointer");
  Obs o;
  if ((s = check_obs(c, obs, &o)) != QF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* dLdE = at<double>(ws_d, c->L.dLdE);
  if ((s = check_loss(loss_kind, E_d, y_d, batch, loss_d, dLdE)) != QF_OK) return s;
  c->call_launches = 0;
  // one prep launch fills the forward's and the backward's tables; the loss
  // rides on the forward's E reduction where the batch allows
  StepLoss sl{loss_kind, y_d, loss_d, dLdE};
  s = fused_forward64(c, c->dt, c->L, theta_d, x_d, batch, o, E_d, ws_d, st, true, &sl);
  if (s != QF_OK) return s;
  if (!sl.done) {
    s = qf_loss64(loss_kind, E_d, y_d, batch, loss_d, dLdE, stream);
    if (s != QF_OK) return s;
    c->call_launches++;
  }
  s = fused_backward64(c, c->dt, c->L, theta_d, x_d, batch, o, dLdE, grad_d, 0, ws_d, st, false);
  c->launches = c->call_launches;
  return s;
}

// The host-buffer step for real inputs of type R (float: complex64 plans,
// double: complex128 plans).
template <class R>
qf_status train_step_host(qf_circuit* c, const R* theta_h, const R* x_h, const R* y_h, int64_t batch,
                          int32_t loss_kind, qf_pauli obs, double* loss_h, double* E_h, double* grad_h, void* ws_d,
                          size_t ws_bytes, void* stream) {
  constexpr bool F64 = sizeof(R) == 8;
  auto step_on = [&](const R* th, const R* xd, const R* yd, void* strm) -> qf_status {
    if constexpr (F64)
      return train_step_eager64(c, th, xd, yd, batch, loss_kind, obs, at<double>(ws_d, c->L.loss),
                                at<double>(ws_d, c->L.E), at<double>(ws_d, c->L.grad), ws_d, ws_bytes, strm);
    else
      return train_step_eager(c, th, xd, yd, batch, loss_kind, obs, at<double>(ws_d, c->L.loss),
                              at<double>(ws_d, c->L.E), at<double>(ws_d, c->L.grad), ws_d, ws_bytes, strm);
  };
  auto step = [&](const R* th, const R* xd, const R* yd) -> qf_status { return step_on(th, xd, yd, stream); };
  qf_status s = check_call(c, batch, ws_d, ws_bytes, F64);
  if (s != QF_OK) return s;
  if (!c->staging) return fail(QF_ERR_UNSUPPORTED, "the plan was made with no_host_staging");
  if ((!theta_h && c->circ.n_params > 0) || (!x_h && batch > 0) || !loss_h || (!grad_h && c->circ.n_params > 0) ||
      (loss_kind == QF_LOSS_MSE && batch > 0 && !y_h))
    return fail(QF_ERR_INVALID_ARG, "null host pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout& L = c->L;
  R* th = at<R>(ws_d, L.theta);
  R* xd = at<R>(ws_d, L.x);
  R* yd = at<R>(ws_d, L.y);
  const int P = c->circ.n_params;
  const bool mse = batch > 0 && loss_kind == QF_LOSS_MSE;
  // Small steps: inputs and outputs each cross the bus as one copy through a
  // pinned staging buffer laid out like the workspace regions (theta, x, y)
  // and (E, dL/dE, grad, loss); large inputs are copied directly.
  const size_t in_span = L.y + (size_t)batch * sizeof(R) - L.theta, out_span = L.loss + 8 - L.E;
  const size_t need = std::max(in_span, out_span);
  if (need <= ((size_t)1 << 20) && !c->h_stage) {
    if (cudaHostAlloc(&c->h_stage, need, cudaHostAllocDefault) == cudaSuccess) {
      c->h_stage_bytes = need;
    } else {
      c->h_stage = nullptr;  // fall back to direct copies
      cudaGetLastError();
    }
  }
  if (c->h_stage && need <= c->h_stage_bytes) {
    char* h = static_cast<char*>(c->h_stage);
    if (P) memcpy(h, theta_h, (size_t)P * sizeof(R));
    if (batch) memcpy(h + (L.x - L.theta), x_h, x_bytes(c, batch));
    if (mse) memcpy(h + (L.y - L.theta), y_h, (size_t)batch * sizeof(R));
    const std::array<uint64_t, 12> key = {(uint64_t)(uintptr_t)ws_d, (uint64_t)ws_bytes, (uint64_t)batch,
                                           (uint64_t)loss_kind, obs.x_mask, obs.z_mask, (uint64_t)(uintptr_t)h,
                                           0, 0, 0, 0, 0};
    auto run = [&](cudaStream_t strm) -> qf_status {
      QF_CU(cudaMemcpyAsync(th, h, in_span, cudaMemcpyHostToDevice, strm));
      const qf_status r = step_on(th, xd, yd, strm);
      if (r != QF_OK) return r;
      QF_CU(cudaMemcpyAsync(h, at<double>(ws_d, L.E), out_span, cudaMemcpyDeviceToHost, strm));
      return QF_OK;
    };
    s = batch > 0 ? graph_step(c, c->hg, key, st, run) : run(st);
    if (s != QF_OK) return s;
    QF_CU(cudaStreamSynchronize(st));
    memcpy(loss_h, h + (L.loss - L.E), 8);
    if (E_h && batch) memcpy(E_h, h, (size_t)batch * 8);
    if (P) memcpy(grad_h, h + (L.grad - L.E), (size_t)P * 8);
    return QF_OK;
  }
  if (P) QF_CU(cudaMemcpyAsync(th, theta_h, (size_t)P * sizeof(R), cudaMemcpyHostToDevice, st));
  if (batch) QF_CU(cudaMemcpyAsync(xd, x_h, x_bytes(c, batch), cudaMemcpyHostToDevice, st));
  if (mse) QF_CU(cudaMemcpyAsync(yd, y_h, (size_t)batch * sizeof(R), cudaMemcpyHostToDevice, st));
  s = step(th, xd, yd);
  if (s != QF_OK) return s;
  QF_CU(cudaMemcpyAsync(loss_h, at<double>(ws_d, L.loss), 8, cudaMemcpyDeviceToHost, st));
  if (E_h && batch) QF_CU(cudaMemcpyAsync(E_h, at<double>(ws_d, L.E), (size_t)batch * 8, cudaMemcpyDeviceToHost, st));
  if (P) QF_CU(cudaMemcpyAsync(grad_h, at<double>(ws_d, L.grad), (size_t)P * 8, cudaMemcpyDeviceToHost, st));
  QF_CU(cudaStreamSynchronize(st));
  return QF_OK;
}

}  // namespace

// A double as two int32 words (low, high) of its bit pattern.
static void push_double(std::vector<int32_t>& w, double v) {
  int32_t b[2];
  memcpy(b, &v, sizeof(v));
  w.push_back(b[0]);
  w.push_back(b[1]);
}

extern "C" {

qf_status qf_plan_export(const qf_circuit* c, int32_t direction, int32_t* buf, int64_t cap, int64_t* len) {
  if (!c || !len) return fail(QF_ERR_INVALID_ARG, "null argument");
  if (!c->planned || c->path != QF_PATH_FUSED) return fail(QF_ERR_WORKSPACE, "no fused plan");
  if (direction < 0 || direction > 2) return fail(QF_ERR_INVALID_ARG, "direction must be 0, 1 or 2");
  const qf::FusedPlan& P = c->fp;
  if (direction == 2) {
    if (P.ckpt_mode != 1) return fail(QF_ERR_INVALID_ARG, "direction 2 needs a ckpt_mode 1 plan");
    std::vector<int32_t> w;
    w.push_back(P.rounds ? 1 : 0);
    w.push_back(P.qshift);
    w.push_back((int32_t)P.a_sched.size());
    for (size_t i = 0; i < P.a_sched.size(); ++i) {
      const qf::PassDesc& pd = P.a_sched[i];
      w.push_back(P.a_dir[i]);
      const int32_t hdr[11] = {pd.op_begin, pd.op_end, pd.psi_src, pd.psi_dst, pd.lam_src, pd.lam_dst,
                               pd.flags, pd.K, pd.n_groups, (int32_t)pd.outer_mask, (int32_t)pd.xm_local};
      w.insert(w.end(), hdr, hdr + 11);
      for (int j = 0; j < 16; ++j) w.push_back(pd.gmap[j]);
      for (int g = 0; g < 4; ++g)
        for (int r = 0; r < 4; ++r) w.push_back(pd.groups[g][r]);
    }
    *len = (int64_t)w.size();
    if (buf) memcpy(buf, w.data(), sizeof(int32_t) * (size_t)std::min<int64_t>(cap, *len));
    return QF_OK;
  }
  const auto& passes = direction == 0 ? P.fwd : P.bwd;
  const auto& ops = direction == 0 ? P.fwd_ops : P.bwd_ops;
  std::vector<int32_t> w;
  w.push_back(P.rounds ? 1 : 0);
  w.push_back(P.qshift);
  w.push_back((int32_t)passes.size());
  for (const qf::PassDesc& pd : passes) {
    const int32_t hdr[11] = {pd.op_begin, pd.op_end, pd.psi_src, pd.psi_dst, pd.lam_src, pd.lam_dst,
                             pd.flags, pd.K, pd.n_groups, (int32_t)pd.outer_mask, (int32_t)pd.xm_local};
    w.insert(w.end(), hdr, hdr + 11);
    for (int j = 0; j < 16; ++j) w.push_back(pd.gmap[j]);
    for (int g = 0; g < 4; ++g)
      for (int r = 0; r < 4; ++r) w.push_back(pd.groups[g][r]);
  }
  w.push_back((int32_t)(ops.size() / 2));
  for (uint32_t v : ops) w.push_back((int32_t)v);
  const int nf = (int)P.fuse_off.size() - 1;
  w.push_back(nf);
  for (int m = 0; m < nf; ++m) {
    w.push_back(P.fuse_off[m + 1] - P.fuse_off[m]);
    for (int j = P.fuse_off[m]; j < P.fuse_off[m + 1]; ++j) {
      w.push_back(P.fuse_gates[j].kind);
      w.push_back(P.fuse_gates[j].param);
      push_double(w, P.fuse_gates[j].angle);
    }
  }
  if (direction == 0) {
    w.push_back((int32_t)P.fwd_rounds.size());
    for (uint32_t v : P.fwd_rounds) w.push_back((int32_t)v);
  } else {
    w.push_back((int32_t)P.bwd_rounds.size());
    for (int32_t v : P.bwd_rounds) w.push_back(v);
  }
  w.push_back(P.n_terms);
  for (int t = 0; t < P.n_terms; ++t) {
    w.push_back(P.term_kind[t]);
    w.push_back(P.term_off[t + 1] - P.term_off[t]);
    for (int j = P.term_off[t]; j < P.term_off[t + 1]; ++j) w.push_back(P.term_params[j]);
    push_double(w, P.term_const[t]);
  }
  *len = (int64_t)w.size();
  if (buf) memcpy(buf, w.data(), sizeof(int32_t) * (size_t)std::min<int64_t>(cap, (int64_t)w.size()));
  return QF_OK;
}

qf_status qf_forward(qf_circuit* c, const float* theta_d, const float* x_d, int64_t batch, qf_pauli obs,
                     double* E_d, void* ws_d, size_t ws_bytes, void* stream) {
  qf_status s = check_call(c, batch, ws_d, ws_bytes);
  if (s != QF_OK) return s;
  if ((!theta_d && c->circ.n_params > 0) || (!x_d && batch > 0) || (!E_d && batch > 0))
    return fail(QF_ERR_INVALID_ARG, "null data pointer");
  Obs o;
  if ((s = check_obs(c, obs, &o)) != QF_OK) return s;
  c->call_launches = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = c->path == QF_PATH_FUSED ? fused_forward(c, c->dt, c->L, theta_d, x_d, batch, o, E_d, ws_d, st)
                               : pg_forward(c, c->dt, c->L, theta_d, x_d, batch, o, E_d, ws_d, st);
  c->launches = c->call_launches;
  return s;
}

qf_status qf_backward(qf_circuit* c, const float* theta_d, const float* x_d, int64_t batch, qf_pauli obs,
                      const double* dLdE_d, double* grad_d, int32_t per_sample, void* ws_d, size_t ws_bytes,
                      void* stream) {
  qf_status s = check_call(c, batch, ws_d, ws_bytes);
  if (s != QF_OK) return s;
  if ((!theta_d && c->circ.n_params > 0) || (!dLdE_d && batch > 0) || (!grad_d && c->circ.n_params > 0))
    return fail(QF_ERR_INVALID_ARG, "null data pointer");
  if (!x_d && batch > 0 && c->encoding == QF_ENC_STATE_IN && c->path == QF_PATH_FUSED && c->fp.ckpt_mode == 1)
    return fail(QF_ERR_INVALID_ARG, "checkpoint mode 1 re-runs the forward from the given states: x_d is needed");
  Obs o;
  if ((s = check_obs(c, obs, &o)) != QF_OK) return s;
  c->call_launches = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = c->path == QF_PATH_FUSED
          ? fused_backward(c, c->dt, c->L, theta_d, x_d, batch, o, dLdE_d, grad_d, per_sample, ws_d, st)
          : pg_backward(c, c->dt, c->L, theta_d, batch, o, dLdE_d, grad_d, per_sample, ws_d, st);
  c->launches += c->call_launches;
  return s;
}

qf_status qf_loss(int32_t kind, const double* E_d, const float* y_d, int64_t batch, double* loss_d,
                  double* dLdE_d, void* stream) {
  const qf_status s = check_loss(kind, E_d, y_d, batch, loss_d, dLdE_d);
  if (s != QF_OK) return s;
  QF_CU(qf::launch_loss(kind, E_d, y_d, batch, loss_d, dLdE_d, static_cast<cudaStream_t>(stream)));
  return QF_OK;
}

qf_status qf_train_step(qf_circuit* c, const float* theta_d, const float* x_d, const float* y_d, int64_t batch,
                        int32_t loss_kind, qf_pauli obs, double* loss_d, double* E_d, double* grad_d, void* ws_d,
                        size_t ws_bytes, void* stream) {
  auto run = [&](cudaStream_t st) {
    return train_step_eager(c, theta_d, x_d, y_d, batch, loss_kind, obs, loss_d, E_d, grad_d, ws_d, ws_bytes, st);
  };
  if (!c || !c->planned || c->path != QF_PATH_FUSED || batch <= 0) return run(static_cast<cudaStream_t>(stream));
  return graph_step(c, c->dg, step_key(theta_d, x_d, y_d, batch, loss_kind, obs, loss_d, E_d, grad_d, ws_d, ws_bytes),
                    static_cast<cudaStream_t>(stream), run);
}

qf_status qf_train_step_host(qf_circuit* c, const float* theta_h, const float* x_h, const float* y_h,
                             int64_t batch, int32_t loss_kind, qf_pauli obs, double* loss_h, double* E_h,
                             double* grad_h, void* ws_d, size_t ws_bytes, void* stream) {
  return train_step_host(c, theta_h, x_h, y_h, batch, loss_kind, obs, loss_h, E_h, grad_h, ws_d, ws_bytes, stream);
}

qf_status qf_train_step_noalloc(qf_circuit* c, const float* theta_d, const float* x_d, const float* y_d,
                                int64_t batch, int32_t loss_kind, qf_pauli obs, double* loss_d, double* E_d,
                                double* grad_d, void* stream) {
  if (!c) return fail(QF_ERR_INVALID_ARG, "null circuit");
  if (!c->planned) return fail(QF_ERR_WORKSPACE, "circuit has no plan (call qf_plan, host_only is enough)");
  if (check_precision(c, false) != QF_OK) return QF_ERR_INVALID_ARG;
  if (batch < 0 || batch > c->batch) return fail(QF_ERR_INVALID_ARG, "batch exceeds the planned batch");
  // one sample's state alone must fit in the block (this also keeps the
  // layout's byte counts far from overflow for any planned batch)
  const size_t state_bytes = (size_t)8 << n_eff_of(c);
  if (batch > 0 && (size_t)batch > (size_t)QF_NOALLOC_MAX_BYTES / state_bytes)
    return fail(QF_ERR_WORKSPACE, "qf_train_step_noalloc: " + std::to_string(batch) + " samples of " +
                                      std::to_string(state_bytes) + " bytes each exceed the fixed " +
                                      std::to_string((size_t)QF_NOALLOC_MAX_BYTES) +
                                      " bytes (QF_NOALLOC_MAX_BYTES); use a smaller batch or qf_train_step");
  if (loss_kind != QF_LOSS_SUM && loss_kind != QF_LOSS_MSE) return fail(QF_ERR_INVALID_ARG, "unknown loss");
  if ((!theta_d && c->circ.n_params > 0) || (batch > 0 && (!x_d || !E_d)) || !loss_d ||
      (!grad_d && c->circ.n_params > 0) || (loss_kind == QF_LOSS_MSE && batch > 0 && !y_d))
    return fail(QF_ERR_INVALID_ARG, "null data pointer");
  Obs o;
  qf_status s = check_obs(c, obs, &o);
  if (s != QF_OK) return s;
  // buffers for this batch behind the plan tables, all inside the fixed block
  const Layout L = make_layout(c, batch);
  const size_t tbytes = c->blob.size();
  const size_t need = tbytes + L.total;
  if (need > (size_t)QF_NOALLOC_MAX_BYTES)
    return fail(QF_ERR_WORKSPACE, "qf_train_step_noalloc needs " + std::to_string(need) +
                                      " bytes of scratch for this circuit and batch, more than the fixed " +
                                      std::to_string((size_t)QF_NOALLOC_MAX_BYTES) +
                                      " (QF_NOALLOC_MAX_BYTES); use a smaller batch or qf_train_step");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QF_ERR_CUDA, std::string("pending CUDA error: ") + cudaGetErrorString(e));
  void* scratch = nullptr;
  size_t cap = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  QF_CU(qf::noalloc_scratch(st, &scratch, &cap));
  QF_CU(cudaMemcpyAsync(scratch, c->blob.data(), tbytes, cudaMemcpyHostToDevice, st));
  const DevTables T = tables_at(c, scratch);
  void* ws = static_cast<char*>(scratch) + tbytes;
  c->call_launches = 0;
  s = c->path == QF_PATH_FUSED ? fused_forward(c, T, L, theta_d, x_d, batch, o, E_d, ws, st)
                               : pg_forward(c, T, L, theta_d, x_d, batch, o, E_d, ws, st);
  if (s != QF_OK) return s;
  double* dLdE = at<double>(ws, L.dLdE);
  QF_CU(qf::launch_loss(loss_kind, E_d, y_d, batch, loss_d, dLdE, st));
  c->call_launches++;
  s = c->path == QF_PATH_FUSED ? fused_backward(c, T, L, theta_d, x_d, batch, o, dLdE, grad_d, 0, ws, st)
                               : pg_backward(c, T, L, theta_d, batch, o, dLdE, grad_d, 0, ws, st);
  c->launches = c->call_launches;
  return s;
}

// ---- complex128 plans ---------------------------------------------------------------
qf_status qf_forward64(qf_circuit* c, const double* theta_d, const double* x_d, int64_t batch, qf_pauli obs,
                       double* E_d, void* ws_d, size_t ws_bytes, void* stream) {
  qf_status s = check_call(c, batch, ws_d, ws_bytes, true);
  if (s != QF_OK) return s;
  if ((!theta_d && c->circ.n_params > 0) || (!x_d && batch > 0) || (!E_d && batch > 0))
    return fail(QF_ERR_INVALID_ARG, "null data pointer");
  Obs o;
  if ((s = check_obs(c, obs, &o)) != QF_OK) return s;
  c->call_launches = 0;
  s = fused_forward64(c, c->dt, c->L, theta_d, x_d, batch, o, E_d, ws_d, static_cast<cudaStream_t>(stream));
  c->launches = c->call_launches;
  return s;
}

qf_status qf_backward64(qf_circuit* c, const double* theta_d, const double* x_d, int64_t batch, qf_pauli obs,
                        const double* dLdE_d, double* grad_d, int32_t per_sample, void* ws_d, size_t ws_bytes,
                        void* stream) {
  qf_status s = check_call(c, batch, ws_d, ws_bytes, true);
  if (s != QF_OK) return s;
  if ((!theta_d && c->circ.n_params > 0) || (!dLdE_d && batch > 0) || (!grad_d && c->circ.n_params > 0))
    return fail(QF_ERR_INVALID_ARG, "null data pointer");
  if (!x_d && batch > 0 && c->encoding == QF_ENC_STATE_IN && c->fp.ckpt_mode == 1)
    return fail(QF_ERR_INVALID_ARG, "checkpoint mode 1 re-runs the forward from the given states: x_d is needed");
  Obs o;
  if ((s = check_obs(c, obs, &o)) != QF_OK) return s;
  c->call_launches = 0;
  s = fused_backward64(c, c->dt, c->L, theta_d, x_d, batch, o, dLdE_d, grad_d, per_sample, ws_d,
                       static_cast<cudaStream_t>(stream));
  c->launches += c->call_launches;
  return s;
}

qf_status qf_loss64(int32_t kind, const double* E_d, const double* y_d, int64_t batch, double* loss_d,
                    double* dLdE_d, void* stream) {
  const qf_status s = check_loss(kind, E_d, y_d, batch, loss_d, dLdE_d);
  if (s != QF_OK) return s;
  QF_CU(qf::launch_loss64(kind, E_d, y_d, batch, loss_d, dLdE_d, static_cast<cudaStream_t>(stream)));
  return QF_OK;
}

qf_status qf_train_step64(qf_circuit* c, const double* theta_d, const double* x_d, const double* y_d,
                          int64_t batch, int32_t loss_kind, qf_pauli obs, double* loss_d, double* E_d,
                          double* grad_d, void* ws_d, size_t ws_bytes, void* stream) {
  auto run = [&](cudaStream_t st) {
    return train_step_eager64(c, theta_d, x_d, y_d, batch, loss_kind, obs, loss_d, E_d, grad_d, ws_d, ws_bytes, st);
  };
  if (!c || !c->planned || batch <= 0) return run(static_cast<cudaStream_t>(stream));
  return graph_step(c, c->dg, step_key(theta_d, x_d, y_d, batch, loss_kind, obs, loss_d, E_d, grad_d, ws_d, ws_bytes),
                    static_cast<cudaStream_t>(stream), run);
}

qf_status qf_train_step_host64(qf_circuit* c, const double* theta_h, const double* x_h, const double* y_h,
                               int64_t batch, int32_t loss_kind, qf_pauli obs, double* loss_h, double* E_h,
                               double* grad_h, void* ws_d, size_t ws_bytes, void* stream) {
  return train_step_host(c, theta_h, x_h, y_h, batch, loss_kind, obs, loss_h, E_h, grad_h, ws_d, ws_bytes, stream);
}

}  // extern "C"

// ---- batched persistent launch over many circuits ---------------------------------
struct qf_batch {
  int n = 0;
  std::vector<qf_circuit*> circ;
  std::vector<int64_t> B;
  std::vector<int64_t> theta_off, x_off, sample_off, grad_off;  // n + 1 each
  std::vector<size_t> ws_off;
  int32_t loss_kind = QF_LOSS_SUM;
  size_t ws_total = 0, lterm_off = 0, queue_off = 0;
  void* d_tables = nullptr;
  qf::BatchArgs args{};
  int64_t prep_total = 0, n_grad_out = 0;
  int grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

template <class T>
T* rel(size_t off) {  // a workspace-relative pointer (rebased by the kernels)
  return reinterpret_cast<T*>(static_cast<uintptr_t>(off));
}

void batch_free(qf_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_tables) cudaFree(b->d_tables);
  b->exec = nullptr;
  b->graph = nullptr;
  b->d_tables = nullptr;
}

}  // namespace

extern "C" {

qf_status qf_batch_create(int32_t n_circuits, qf_circuit* const* circuits, const int64_t* batch,
                          const qf_pauli* obs, int32_t loss_kind, size_t* workspace_bytes, qf_batch** out) {
  if (!out || !workspace_bytes) return fail(QF_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (n_circuits <= 0 || !circuits || !batch || !obs) return fail(QF_ERR_INVALID_ARG, "empty or null circuit list");
  if (loss_kind != QF_LOSS_SUM && loss_kind != QF_LOSS_MSE) return fail(QF_ERR_INVALID_ARG, "unknown loss");
  qf_batch* b = nullptr;
  try {
    b = new qf_batch();
    b->n = n_circuits;
    b->loss_kind = loss_kind;
    b->circ.assign(circuits, circuits + n_circuits);
    b->B.assign(batch, batch + n_circuits);
    b->theta_off.assign(n_circuits + 1, 0);
    b->x_off.assign(n_circuits + 1, 0);
    b->sample_off.assign(n_circuits + 1, 0);
    b->grad_off.assign(n_circuits + 1, 0);
    b->ws_off.assign(n_circuits, 0);
    std::vector<Layout> lay(n_circuits);
    std::vector<Obs> ob(n_circuits);
    size_t ws = 0;
    for (int i = 0; i < n_circuits; ++i) {
      qf_circuit* c = b->circ[i];
      const std::string at = " (circuit " + std::to_string(i) + ")";
      if (!c || !c->planned) throw std::invalid_argument("circuit has no plan" + at);
      if (c->encoding != QF_ENC_RY_X) throw std::invalid_argument("batched launches take RY(x) encodings" + at);
      if (c->f64) throw std::invalid_argument("batched launches are complex64" + at);
      if (c->path == QF_PATH_FUSED && c->fp.has_rx)
        throw std::invalid_argument("batched launches take RZ/RY round programs (no RX)" + at);
      if (c->path == QF_PATH_FUSED && (c->fp.ckpt_mode != 0 || c->tc))
        throw std::invalid_argument("batched launches use checkpoint mode 0 on the CUDA cores" + at);
      if (c->path != QF_PATH_FUSED || !c->fp.rounds)
        throw std::invalid_argument("batched launches need fused round programs (RZ/RY rotations, CZ on "
                                    "neighbouring qubits, at least 7 qubits per tile)" + at);
      if (b->B[i] < 1) throw std::invalid_argument("batch must be >= 1" + at);
      if (check_obs(c, obs[i], &ob[i]) != QF_OK) throw std::invalid_argument(g_err + at);
      for (const qf::PassDesc& pd : c->fp.fwd) {
        uint32_t xl;
        if ((pd.flags & qf::PF_EXPECT) && !local_xmask(pd, ob[i].x, &xl))
          throw std::invalid_argument("observable X/Y qubits must lie in the last pass's tile" + at);
      }
      lay[i] = make_layout(c, b->B[i]);
      b->ws_off[i] = ws;
      ws += lay[i].total;
      b->theta_off[i + 1] = b->theta_off[i] + c->circ.n_params;
      b->x_off[i + 1] = b->x_off[i] + b->B[i] * c->circ.n;
      b->sample_off[i + 1] = b->sample_off[i] + b->B[i];
      b->grad_off[i + 1] = b->grad_off[i] + c->circ.n_params;
    }
    b->lterm_off = ws;
    ws += al((size_t)b->sample_off[n_circuits] * 8);
    b->queue_off = ws;
    ws += 256;
    b->ws_total = ws;

    // ---- device tables: every circuit's plan tables and pass descriptors, the
    // circuit records, the work items and the prefix offsets
    std::vector<size_t> tab_off(n_circuits), fwd_off(n_circuits), bwd_off(n_circuits);
    size_t o = 0;
    for (int i = 0; i < n_circuits; ++i) {
      tab_off[i] = o;
      o = al(o + b->circ[i]->blob.size());
      fwd_off[i] = o;
      o = al(o + b->circ[i]->fp.fwd.size() * sizeof(qf::PassDesc));
      bwd_off[i] = o;
      o = al(o + b->circ[i]->fp.bwd.size() * sizeof(qf::PassDesc));
    }
    // work items: samples of one circuit; largest first
    std::vector<qf::BatchItem> items;
    std::vector<double> cost;
    for (int i = 0; i < n_circuits; ++i) {
      const qf::FusedPlan& P = b->circ[i]->fp;
      const int tps_log2 = P.n_eff - P.K;
      const int tpc = qf::kThreads >> (P.K - qf::kRegBits);
      const int step = tps_log2 == 0 ? tpc : 1;
      for (int64_t b0 = 0; b0 < b->B[i]; b0 += step) {
        items.push_back({i, (int32_t)b0});
        const double ns = (double)std::min<int64_t>(step, b->B[i] - b0);
        cost.push_back(ns * std::ldexp(1.0, P.n_eff) * (double)std::max(P.n_rounds, 1));
      }
    }
    std::vector<size_t> ord(items.size());
    for (size_t k = 0; k < ord.size(); ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    const size_t circ_off = o;
    o = al(o + n_circuits * sizeof(qf::BatchCircuit));
    const size_t items_off = o;
    o = al(o + items.size() * sizeof(qf::BatchItem));
    const size_t prep_off = o;
    o = al(o + (n_circuits + 1) * sizeof(int64_t));
    const size_t gout_off = o;
    o = al(o + (n_circuits + 1) * sizeof(int64_t));
    const size_t total = o;

    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return fail(QF_ERR_OOM, std::string("cudaMalloc of batch tables failed: ") + cudaGetErrorString(e));
    }
    b->d_tables = d;
    char* base = static_cast<char*>(d);
    std::vector<char> img(total, 0);
    std::vector<qf::BatchCircuit> recs(n_circuits);
    std::vector<int64_t> prep_pref(n_circuits + 1, 0), gout_pref(n_circuits + 1, 0);
    for (int i = 0; i < n_circuits; ++i) {
      qf_circuit* c = b->circ[i];
      const qf::FusedPlan& P = c->fp;
      const Layout& L = lay[i];
      const size_t w0 = b->ws_off[i];
      memcpy(img.data() + tab_off[i], c->blob.data(), c->blob.size());
      std::vector<qf::PassDesc> fp = P.fwd, bp = P.bwd;
      for (auto& pd : fp) {
        pd.xm_local = 0;
        if (pd.flags & qf::PF_EXPECT) local_xmask(pd, ob[i].x, &pd.xm_local);
      }
      for (auto& pd : bp) {
        pd.xm_local = 0;
        if (pd.lam_src == qf::LAM_SEED) local_xmask(pd, ob[i].x, &pd.xm_local);
      }
      memcpy(img.data() + fwd_off[i], fp.data(), fp.size() * sizeof(qf::PassDesc));
      memcpy(img.data() + bwd_off[i], bp.data(), bp.size() * sizeof(qf::PassDesc));
      const DevTables T = tables_at(c, base + tab_off[i]);
      qf::BatchCircuit& r = recs[i];
      qf::PassArgs a{};
      a.n_eff = P.n_eff;
      a.tps_log2 = P.n_eff - P.K;
      a.B = b->B[i];
      a.mats = rel<const float4>(w0 + L.mats);
      a.enc = rel<const float2>(w0 + L.enc);
      a.work = rel<float2>(w0 + L.work);
      a.lam = rel<float2>(w0 + L.lam);
      a.slots = rel<float2>(w0 + L.slots);
      a.slot_stride = L.state_elems;
      a.z_mask = ob[i].z;
      a.y_count = ob[i].y;
      a.dLdE = rel<const double>(w0 + L.dLdE);
      a.e_part = rel<double>(w0 + L.epart);
      a.g_part = rel<double>(w0 + L.gpart);
      a.n_slots = P.n_terms;
      r.fa = a;
      r.fa.ops = T.fwd_ops;
      r.fa.rounds = T.fwd_rounds;
      r.fa.rpar = rel<const float4>(w0 + L.rpf);
      r.ba = a;
      r.ba.ops = T.bwd_ops;
      r.ba.rounds = T.bwd_rounds;
      r.ba.rpar = rel<const float4>(w0 + L.rpb);
      r.ba.g_accum = a.tps_log2 > 0 ? 1 : 0;
      r.fwd = reinterpret_cast<const qf::PassDesc*>(base + fwd_off[i]);
      r.bwd = reinterpret_cast<const qf::PassDesc*>(base + bwd_off[i]);
      r.n_fwd = (int32_t)fp.size();
      r.n_bwd = (int32_t)bp.size();
      r.samples_per_item = a.tps_log2 == 0 ? (qf::kThreads >> (P.K - qf::kRegBits)) : 1;
      r.loss_kind = loss_kind;
      r.inv_B = 1.0 / (double)b->B[i];
      r.theta_off = b->theta_off[i];
      r.x_off = b->x_off[i];
      r.sample_off = b->sample_off[i];
      r.grad_off = b->grad_off[i];
      qf::PrepArgs& p = r.prep;
      p = qf::PrepArgs{};
      p.n_fused = P.rounds ? 0 : (int32_t)P.fuse_off.size() - 1;  // round tables only
      p.fuse_off = T.fuse_off;
      p.fuse_gates = T.fuse_gates;
      p.mats = rel<float4>(w0 + L.mats);
      p.n_terms = 0;  // round programs: the round tables hold every angle
      p.term_off = T.term_off;
      p.term_params = T.term_params;
      p.term_const = T.term_const;
      p.B = b->B[i];
      p.n = c->circ.n;
      p.n_eff = P.n_eff;
      p.qshift = P.qshift;
      p.enc = rel<float2>(w0 + L.enc);
      p.n_rpf = (int32_t)(P.fwd_rounds.size() / qf::kFwdRoundWords);
      p.rpf_src = T.fwd_rounds;
      p.rpf_terms = T.fwd_rterms;
      p.rpf = rel<float4>(w0 + L.rpf);
      p.n_rpb = (int32_t)(P.bwd_rounds.size() / qf::kBwdRoundWords);
      p.rpb_src = T.bwd_rounds;
      p.rpb_terms = T.bwd_rterms;
      p.rpb = rel<float4>(w0 + L.rpb);
      r.n_params = c->circ.n_params;
      r.param_off = T.param_off;
      r.param_terms = T.param_terms;
      prep_pref[i + 1] = prep_pref[i] + p.n_fused + p.n_terms + p.B * p.n_eff + qf::round_par_elems(p);
      gout_pref[i + 1] = gout_pref[i] + c->circ.n_params;
    }
    memcpy(img.data() + circ_off, recs.data(), recs.size() * sizeof(qf::BatchCircuit));
    for (size_t k = 0; k < ord.size(); ++k)
      memcpy(img.data() + items_off + k * sizeof(qf::BatchItem), &items[ord[k]], sizeof(qf::BatchItem));
    memcpy(img.data() + prep_off, prep_pref.data(), prep_pref.size() * sizeof(int64_t));
    memcpy(img.data() + gout_off, gout_pref.data(), gout_pref.size() * sizeof(int64_t));
    e = cudaMemcpy(d, img.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      batch_free(b);
      delete b;
      return fail(QF_ERR_CUDA, std::string("batch table upload failed: ") + cudaGetErrorString(e));
    }
    b->args = qf::BatchArgs{};
    b->args.circ = reinterpret_cast<const qf::BatchCircuit*>(base + circ_off);
    b->args.n_circ = n_circuits;
    b->args.items = reinterpret_cast<const qf::BatchItem*>(base + items_off);
    b->args.n_items = (int32_t)items.size();
    b->args.prep_off = reinterpret_cast<const int64_t*>(base + prep_off);
    b->args.grad_out_off = reinterpret_cast<const int64_t*>(base + gout_off);
    b->args.n_samples = b->sample_off[n_circuits];
    b->prep_total = prep_pref[n_circuits];
    b->n_grad_out = gout_pref[n_circuits];
    b->grid = qf::batch_grid();
    if (b->grid <= 0) {
      batch_free(b);
      delete b;
      return fail(QF_ERR_CUDA, "cannot query the device's SM count");
    }
  } catch (const std::bad_alloc&) {
    if (b) {
      batch_free(b);
      delete b;
    }
    return fail(QF_ERR_OOM, "host allocation failed");
  } catch (const std::exception& ex) {
    if (b) {
      batch_free(b);
      delete b;
    }
    return fail(QF_ERR_INVALID_ARG, ex.what());
  }
  *workspace_bytes = b->ws_total;
  *out = b;
  return QF_OK;
}

qf_status qf_batch_layout(const qf_batch* b, int64_t* theta_off, int64_t* x_off, int64_t* sample_off) {
  if (!b) return fail(QF_ERR_INVALID_ARG, "null batch");
  const size_t n = (size_t)b->n + 1;
  if (theta_off) memcpy(theta_off, b->theta_off.data(), n * sizeof(int64_t));
  if (x_off) memcpy(x_off, b->x_off.data(), n * sizeof(int64_t));
  if (sample_off) memcpy(sample_off, b->sample_off.data(), n * sizeof(int64_t));
  return QF_OK;
}

qf_status qf_batch_train_step(qf_batch* b, const float* theta_d, const float* x_d, const float* y_d,
                              double* loss_d, double* E_d, double* grad_d, void* ws_d, size_t ws_bytes,
                              void* stream) {
  if (!b) return fail(QF_ERR_INVALID_ARG, "null batch");
  if (!ws_d || ((uintptr_t)ws_d & 255) != 0) return fail(QF_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < b->ws_total) return fail(QF_ERR_WORKSPACE, "workspace smaller than qf_batch_create reported");
  if (!theta_d || !x_d || !loss_d || !E_d || !grad_d || (b->loss_kind == QF_LOSS_MSE && !y_d))
    return fail(QF_ERR_INVALID_ARG, "null data pointer");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QF_ERR_CUDA, std::string("pending CUDA error: ") + cudaGetErrorString(e));
  qf::BatchArgs a = b->args;
  a.ws = static_cast<char*>(ws_d);
  a.theta = theta_d;
  a.x = x_d;
  a.y = y_d;
  a.E = E_d;
  a.grad = grad_d;
  a.loss = loss_d;
  a.lterm = reinterpret_cast<double*>(a.ws + b->lterm_off);
  a.queue = reinterpret_cast<int32_t*>(a.ws + b->queue_off);
  QF_CU(qf::launch_batch(a, b->grid, b->prep_total, b->n_grad_out, static_cast<cudaStream_t>(stream)));
  return QF_OK;
}

qf_status qf_batch_graph_capture(qf_batch* b, const float* theta_d, const float* x_d, const float* y_d,
                                 double* loss_d, double* E_d, double* grad_d, void* ws_d, size_t ws_bytes,
                                 void* stream) {
  if (!b) return fail(QF_ERR_INVALID_ARG, "null batch");
  if (!stream) return fail(QF_ERR_INVALID_ARG, "capture needs a non-default stream");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  // one eager step first: per-device kernel attributes are set outside the capture
  qf_status s = qf_batch_train_step(b, theta_d, x_d, y_d, loss_d, E_d, grad_d, ws_d, ws_bytes, stream);
  if (s != QF_OK) return s;
  QF_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  s = qf_batch_train_step(b, theta_d, x_d, y_d, loss_d, E_d, grad_d, ws_d, ws_bytes, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s != QF_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return fail(QF_ERR_CUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
  b->graph = g;
  QF_CU(cudaGraphInstantiate(&b->exec, g, 0));
  return QF_OK;
}

qf_status qf_batch_graph_launch(qf_batch* b, void* stream) {
  if (!b || !b->exec) return fail(QF_ERR_INVALID_ARG, "no captured graph (call qf_batch_graph_capture)");
  QF_CU(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return QF_OK;
}

qf_status qf_batch_info(const qf_batch* b, int64_t* n_items, int64_t* n_samples, int64_t* n_params) {
  if (!b) return fail(QF_ERR_INVALID_ARG, "null batch");
  if (n_items) *n_items = b->args.n_items;
  if (n_samples) *n_samples = b->args.n_samples;
  if (n_params) *n_params = b->n_grad_out;
  return QF_OK;
}

qf_status qf_batch_destroy(qf_batch* b) {
  if (!b) return QF_OK;
  batch_free(b);
  delete b;
  return QF_OK;
}

qf_status qf_profile(qf_circuit* c, int32_t on) {
  if (!c) return fail(QF_ERR_INVALID_ARG, "null circuit");
  if (on && c->ev.empty()) {
    c->ev.resize(2 * kMaxProfilePairs);
    for (auto& e : c->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) {
        e = nullptr;
        destroy_events(c);
        return fail(QF_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(r));
      }
    }
    c->ev_dir.assign(kMaxProfilePairs, 0);
    c->ev_launches.assign(kMaxProfilePairs, 0);
  }
  c->profile = on != 0;
  c->ev_used = 0;
  return QF_OK;
}

qf_status qf_profile_read(qf_circuit* c, double* fwd_ms, int64_t* fwd_launches, double* bwd_ms,
                          int64_t* bwd_launches) {
  if (!c) return fail(QF_ERR_INVALID_ARG, "null circuit");
  double ms[2] = {0, 0};
  int64_t nl[2] = {0, 0};
  for (size_t k = 0; k < c->ev_used; ++k) {
    QF_CU(cudaEventSynchronize(c->ev[2 * k + 1]));
    float t = 0.f;
    QF_CU(cudaEventElapsedTime(&t, c->ev[2 * k], c->ev[2 * k + 1]));
    ms[c->ev_dir[k]] += t;
    nl[c->ev_dir[k]] += c->ev_launches[k];
  }
  c->ev_used = 0;
  if (fwd_ms) *fwd_ms = ms[0];
  if (fwd_launches) *fwd_launches = nl[0];
  if (bwd_ms) *bwd_ms = ms[1];
  if (bwd_launches) *bwd_launches = nl[1];
  return QF_OK;
}

qf_status qf_launch_count(const qf_circuit* c, int64_t* launches) {
  if (!c || !launches) return fail(QF_ERR_INVALID_ARG, "null argument");
  *launches = c->launches;
  return QF_OK;
}

qf_status qf_graph_stats(const qf_circuit* c, int64_t* recorded, int64_t* replayed) {
  if (!c || !recorded || !replayed) return fail(QF_ERR_INVALID_ARG, "null argument");
  *recorded = c->g_recorded;
  *replayed = c->g_replayed;
  return QF_OK;
}

}  // extern "C"
