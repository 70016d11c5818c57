// Complex128 fused forward / adjoint passes for sm_103a.
//
// The same plans and step programs as the complex64 passes (Secs. 3.2-3.3),
// with every amplitude, table entry and partial in float64: the
// double-precision state type the paper's library supports next to
// complex64. Generic steps apply a fused 2x2 per register bit in the forward,
// CZ signs and CNOT swaps, and un-apply one rotation at a time in the
// adjoint. Round programs apply per register bit an RY and a merged RZ run as
// three-shear rotations with pending CZ signs, so a qubit-layer of the
// hardware-efficient ansatz costs 12 FP64 instructions per amplitude pair
// forward (16 as a fused 2x2) and two gradient terms of 16 backward (three of
// 20 one rotation at a time). GB300's FP64 pipe runs at 1/61 of its FP32
// rate, so these passes are bound by FP64 instruction issue, never by memory.
//
// A CTA (256 threads) owns 4096 amplitudes per state, as in the complex64
// passes; the tile is 64 KiB per state here (16-byte amplitudes), so the
// adjoint (psi and lambda) takes 128 KiB. One CTA per SM (8 warps) keeps the
// FP64 pipe busy; the launch bound lets the 16 + 16 double2 registers of the
// adjoint step stay in registers.
//
// Shared-memory layout: amplitude with local index i lives at
// i ^ ((i >> 4) & 7). Eight 16-byte amplitudes fill the 32 banks, and a
// 16-byte access is served eight lanes at a time. Register groups are local
// nibbles: for nibble 0 those eight lanes differ in local bits 4..6, which the
// XOR folds into the low three bits; for any other group they differ in bits
// 0..2 directly. Either way the eight lanes hit eight distinct bank quads.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace qf {
namespace {

__device__ __forceinline__ uint32_t swz64(uint32_t i) { return i ^ ((i >> 4) & 7u); }

// Scatter the low bits of src into the set bits of mask (ascending).
__device__ __forceinline__ uint32_t pdep(uint32_t src, uint32_t mask) {
  uint32_t r = 0;
  for (uint32_t bb = 1; mask; bb <<= 1) {
    const uint32_t low = mask & (0u - mask);
    if (src & bb) r |= low;
    mask ^= low;
  }
  return r;
}

__device__ __forceinline__ uint32_t reg_offset(uint32_t j, const uint32_t (&o)[4]) {
  return ((j & 1u) ? o[0] : 0u) ^ ((j & 2u) ? o[1] : 0u) ^ ((j & 4u) ? o[2] : 0u) ^ ((j & 8u) ? o[3] : 0u);
}

// v with its sign flipped when s = 1
__device__ __forceinline__ double flipd(double v, uint32_t s) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)s << 63));
}

// phase i^k times v
__device__ __forceinline__ double2 ipow(double2 v, uint32_t k) {
  switch (k & 3u) {
    case 0: return v;
    case 1: return make_double2(-v.y, v.x);
    case 2: return make_double2(-v.x, -v.y);
    default: return make_double2(v.y, -v.x);
  }
}

// (a, b) <- (u00 a + u01 b, u10 a + u11 b) on the pairs of register bit R.
template <int R>
__device__ __forceinline__ void apply_u64(double2 (&r)[16], const double2 u00, const double2 u01, const double2 u10,
                                          const double2 u11) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    const double2 x = r[j], y = r[j1];
    r[j].x = u00.x * x.x - u00.y * x.y + u01.x * y.x - u01.y * y.y;
    r[j].y = u00.x * x.y + u00.y * x.x + u01.x * y.y + u01.y * y.x;
    r[j1].x = u10.x * x.x - u10.y * x.y + u11.x * y.x - u11.y * y.y;
    r[j1].y = u10.x * x.y + u10.y * x.x + u11.x * y.y + u11.y * y.x;
  }
}

// Un-apply u = exp(-i phi P / 2) (P = Z, Y or X on register bit R) from psi
// and lambda; returns the thread's sum of Im<lambda|P|psi> over its pairs,
// taken before the un-apply. Re<lambda_j| du/dphi |psi_{j-1}> =
// (1/2) Im<lambda_j|P|psi_j> (Sec. 3.3); the 1/2 is applied at the flush.
template <int R, int KIND>
__device__ __forceinline__ double bwd_gate64(double2 (&p)[16], double2 (&l)[16], const double c, const double s) {
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    const double2 p0 = p[j], p1 = p[j1], l0 = l[j], l1 = l[j1];
    if (KIND == G_RZ) {
      acc += l0.x * p0.y - l0.y * p0.x - l1.x * p1.y + l1.y * p1.x;
      // u^dagger = diag(c + i s, c - i s)
      p[j] = make_double2(c * p0.x - s * p0.y, c * p0.y + s * p0.x);
      p[j1] = make_double2(c * p1.x + s * p1.y, c * p1.y - s * p1.x);
      l[j] = make_double2(c * l0.x - s * l0.y, c * l0.y + s * l0.x);
      l[j1] = make_double2(c * l1.x + s * l1.y, c * l1.y - s * l1.x);
    } else if (KIND == G_RY) {
      acc += l1.x * p0.x + l1.y * p0.y - l0.x * p1.x - l0.y * p1.y;
      // u^dagger = [[c, s], [-s, c]]
      p[j] = make_double2(c * p0.x + s * p1.x, c * p0.y + s * p1.y);
      p[j1] = make_double2(c * p1.x - s * p0.x, c * p1.y - s * p0.y);
      l[j] = make_double2(c * l0.x + s * l1.x, c * l0.y + s * l1.y);
      l[j1] = make_double2(c * l1.x - s * l0.x, c * l1.y - s * l0.y);
    } else {  // RX
      acc += l0.x * p1.y - l0.y * p1.x + l1.x * p0.y - l1.y * p0.x;
      // u^dagger = [[c, i s], [i s, c]]
      p[j] = make_double2(c * p0.x - s * p1.y, c * p0.y + s * p1.x);
      p[j1] = make_double2(c * p1.x - s * p0.y, c * p1.y + s * p0.x);
      l[j] = make_double2(c * l0.x - s * l1.y, c * l0.y + s * l1.x);
      l[j1] = make_double2(c * l1.x - s * l0.y, c * l1.y + s * l0.x);
    }
  }
  return acc;
}

template <int KIND>
__device__ __forceinline__ double bwd_dispatch64(uint32_t r, double2 (&p)[16], double2 (&l)[16], double c,
                                                 double s) {
  switch (r) {
    case 0: return bwd_gate64<0, KIND>(p, l, c, s);
    case 1: return bwd_gate64<1, KIND>(p, l, c, s);
    case 2: return bwd_gate64<2, KIND>(p, l, c, s);
    default: return bwd_gate64<3, KIND>(p, l, c, s);
  }
}

// CNOT with its target on register bit RT: swap the target pairs whose control
// is 1 (register bit cb when creg, else bit cb of the thread's base index gb).
// Self-inverse, so the adjoint applies the same swap to psi and lambda.
template <int RT, bool BWD>
__device__ __forceinline__ void cnot64(double2 (&r)[16], double2 (&l)[16], bool creg, uint32_t cb, uint32_t gb) {
  const uint32_t cg = (gb >> cb) & 1u;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << RT)) continue;
    const int j1 = j | (1 << RT);
    const bool on = creg ? (((uint32_t)j >> cb) & 1u) != 0 : cg != 0;
    const double2 a = r[j], b = r[j1];
    r[j] = on ? b : a;
    r[j1] = on ? a : b;
    if (BWD) {
      const double2 c = l[j], d = l[j1];
      l[j] = on ? d : c;
      l[j1] = on ? c : d;
    }
  }
}

// ---- round programs (the complex64 round programs' items in float64) -----------
// A round applies one item per register bit r (the RY, then the merged RZ
// run; the adjoint runs the exact reverse) and then the round's CZ links.
// Rotations run as three shears: a plane rotation by phi is x += a y;
// y += b x; x += a y with a = -tan(phi/2), b = sin(phi), |a| <= 1 for
// |phi| <= pi/2 (term angles are wrapped into (-pi, pi], the wrap parity
// kept as a sign). Pending CZ signs D: the registers hold psi~ with
// psi = D psi~, D = (-1)^(c0 + sum_r A_r j_r) (bit 4: c0, bits 0..3: A);
// a gate on register bit r sees only Z_r^(A_r), folded into it; CZs between
// two register bits are signs of the round's diagonal table.

// Link q couples qubit q with q + 1 mod n: the constant (t2 & gb) and linear
// (u) parts of the links L for thread base index gb.
__device__ __forceinline__ void link_terms64(uint32_t L, uint32_t gb, int n, uint32_t& t2, uint32_t& u) {
  const uint32_t nmask = n >= 32 ? ~0u : ((1u << n) - 1u);
  const uint32_t t1 = L & gb;
  t2 = L & (((gb >> 1) | ((gb & 1u) << (n - 1))) & nmask);
  u = (((t1 << 1) | (t1 >> (n - 1))) & nmask) ^ t2;
}

__device__ __forceinline__ void chain64(uint32_t L, uint32_t gb, const uint32_t (&p)[4], int n, uint32_t& D) {
  uint32_t t2, u;
  link_terms64(L, gb, n, t2, u);
  D ^= (((u >> p[0]) & 1u) | (((u >> p[1]) & 1u) << 1) | (((u >> p[2]) & 1u) << 2) | (((u >> p[3]) & 1u) << 3)) |
       ((__popc(t2 & gb) & 1u) << 4);
}

// Multiply the registers by D (end of a step).
template <bool BWD>
__device__ __forceinline__ void pending64(uint32_t D, double2 (&r)[16], double2 (&l)[16]) {
  uint32_t S = (D & 16u) ? 0xFFFFu : 0u;
  S ^= (D & 1u) ? 0xAAAAu : 0u;
  S ^= (D & 2u) ? 0xCCCCu : 0u;
  S ^= (D & 4u) ? 0xF0F0u : 0u;
  S ^= (D & 8u) ? 0xFF00u : 0u;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t f = (S >> j) & 1u;
    r[j] = make_double2(flipd(r[j].x, f), flipd(r[j].y, f));
    if (BWD) l[j] = make_double2(flipd(l[j].x, f), flipd(l[j].y, f));
  }
}

// The rotation of a forward item on register bit R (RY, or RX where rx):
// y holds the term's shear parameters of the un-apply direction; applying
// rotates the other way. A pending Z_R turns the rotation by w into one by
// -w; the wrap parity goes to the pending constant sign. An absent rotation
// (no term) is skipped.
template <int R>
__device__ __forceinline__ void rot_fwd64(double2 (&r)[16], const Shear64& y, uint32_t a, uint32_t& D,
                                          bool has_y, bool rx) {
  const double ty = a ? y.t : -y.t, sy = a ? -y.s : y.s;
  if (has_y && rx) {
    // RX(w): a rotation by -w/2 of (re p0, im p1) and (re p1, im p0):
    // x += t y; y -= s x; x += t y (t, s negated under a pending Z_R)
    const double tx = -ty, sx = sy;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & (1 << R)) continue;
      const int j1 = j | (1 << R);
      double2 p0 = r[j], p1 = r[j1];
      p0.x = fma(tx, p1.y, p0.x); p1.y = fma(-sx, p0.x, p1.y); p0.x = fma(tx, p1.y, p0.x);
      p1.x = fma(tx, p0.y, p1.x); p0.y = fma(-sx, p1.x, p0.y); p1.x = fma(tx, p0.y, p1.x);
      r[j] = p0;
      r[j1] = p1;
    }
  } else if (has_y) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & (1 << R)) continue;
      const int j1 = j | (1 << R);
      double2 p0 = r[j], p1 = r[j1];
      // RY(w) on (p0, p1): rotation by +w/2, the same shears on re and im
      p0.x = fma(ty, p1.x, p0.x); p0.y = fma(ty, p1.y, p0.y);
      p1.x = fma(sy, p0.x, p1.x); p1.y = fma(sy, p0.y, p1.y);
      p0.x = fma(ty, p1.x, p0.x); p0.y = fma(ty, p1.y, p0.y);
      r[j] = p0;
      r[j1] = p1;
    }
  }
  D ^= (uint32_t)(y.wrap & 1) << 4;
}

// v *= (c + i s)
__device__ __forceinline__ void cmul64(double2& v, double c, double s) {
  const double x = v.x;
  v.x = fma(c, x, -s * v.y);
  v.y = fma(s, x, c * v.y);
}

// The round's diagonal (its 4 RZ runs and the CZ links between register
// bits, merged), applied: register amplitude j times ph[j]. It commutes with
// the rotations on the other register bits and with the pending signs.
__device__ __forceinline__ void diag64(double2 (&r)[16], const double2* ph) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const double2 e = ph[j];
    cmul64(r[j], e.x, e.y);
  }
}

// Adjoint side of the round's diagonal: g[r] = sum_j sigma_r(j) w_j with
// w_j = Im(conj(lambda_j) psi_j), sigma_r(j) = +1 where bit r of j is clear,
// else -1 (the RZ-run terms; w_j is unchanged by the diagonal, and Z_r
// commutes with the rotations on the other bits), then the un-apply.
__device__ __forceinline__ void diag_bwd64(double2 (&p)[16], double2 (&l)[16], const double2* ph, double (&g)[8]) {
  double s2[4];
  double d0 = 0.0, d1 = 0.0, se = 0.0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    double2& p0 = p[2 * m];
    double2& p1 = p[2 * m + 1];
    double2& l0 = l[2 * m];
    double2& l1 = l[2 * m + 1];
    const double w0 = fma(l0.x, p0.y, -l0.y * p0.x);
    const double w1 = fma(l1.x, p1.y, -l1.y * p1.x);
    const double2 e0 = ph[2 * m], e1 = ph[2 * m + 1];
    cmul64(p0, e0.x, e0.y);
    cmul64(l0, e0.x, e0.y);
    cmul64(p1, e1.x, e1.y);
    cmul64(l1, e1.x, e1.y);
    const double sm = w0 + w1;
    d0 += w0 - w1;
    if (m & 1) {
      s2[m >> 1] = se + sm;
      d1 += se - sm;
    } else {
      se = sm;
    }
  }
  g[0] = d0;
  g[1] = d1;
  g[2] = (s2[0] - s2[1]) + (s2[2] - s2[3]);
  g[3] = (s2[0] + s2[1]) - (s2[2] + s2[3]);
}

// Un-apply one rotation on register bit R by three shears; returns the
// thread's sum of Im<lambda|P|psi> taken before it.
//   RY: (x, y) <- RY(w)^dagger (x, y), a rotation by -w/2: a = t, b = -s.
template <int R, int KIND>
__device__ __forceinline__ double shear_bwd64(double2 (&p)[16], double2 (&l)[16], const double t, const double s) {
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    double2 p0 = p[j], p1 = p[j1], l0 = l[j], l1 = l[j1];
    if (KIND == G_RX) {
      // Im<lambda|X|psi>; RX(w)^dagger rotates (re p0, im p1) and (re p1, im p0) by +w/2
      acc += l0.x * p1.y - l0.y * p1.x + l1.x * p0.y - l1.y * p0.x;
      p0.x = fma(-t, p1.y, p0.x); p1.y = fma(s, p0.x, p1.y); p0.x = fma(-t, p1.y, p0.x);
      p1.x = fma(-t, p0.y, p1.x); p0.y = fma(s, p1.x, p0.y); p1.x = fma(-t, p0.y, p1.x);
      l0.x = fma(-t, l1.y, l0.x); l1.y = fma(s, l0.x, l1.y); l0.x = fma(-t, l1.y, l0.x);
      l1.x = fma(-t, l0.y, l1.x); l0.y = fma(s, l1.x, l0.y); l1.x = fma(-t, l0.y, l1.x);
    } else {
      acc += l1.x * p0.x + l1.y * p0.y - l0.x * p1.x - l0.y * p1.y;
      p0.x = fma(t, p1.x, p0.x); p0.y = fma(t, p1.y, p0.y);
      p1.x = fma(-s, p0.x, p1.x); p1.y = fma(-s, p0.y, p1.y);
      p0.x = fma(t, p1.x, p0.x); p0.y = fma(t, p1.y, p0.y);
      l0.x = fma(t, l1.x, l0.x); l0.y = fma(t, l1.y, l0.y);
      l1.x = fma(-s, l0.x, l1.x); l1.y = fma(-s, l0.y, l1.y);
      l0.x = fma(t, l1.x, l0.x); l0.y = fma(t, l1.y, l0.y);
    }
    p[j] = p0;
    p[j1] = p1;
    l[j] = l0;
    l[j1] = l1;
  }
  return acc;
}

// The rotation of an adjoint item on register bit R, un-applied after the
// round's diagonal; gy: its Im<lambda|P|psi>. With a pending Z_R it
// un-applies as the rotation by +w and gy changes sign. An absent rotation is
// skipped; its value is 0.
template <int R>
__device__ __forceinline__ void rot_bwd64(double2 (&p)[16], double2 (&l)[16], const Shear64& y, uint32_t a,
                                          uint32_t& D, double& gy, bool has_y, bool rx) {
  gy = 0.0;
  if (has_y) {
    const double t = a ? -y.t : y.t, s = a ? -y.s : y.s;
    const double g = rx ? shear_bwd64<R, G_RX>(p, l, t, s) : shear_bwd64<R, G_RY>(p, l, t, s);
    gy = a ? -g : g;
  }
  D ^= (uint32_t)(y.wrap & 1) << 4;
}

// Reduce 8 per-thread values over `lanes` lanes (8, 16 or 32; whole-warp
// call): afterwards the lanes with (lane & (lanes/8 - 1)) == 0 hold the 8
// lanes-sums, lane's being that of value *idx.
__device__ __forceinline__ double butterfly8_64(double (&v)[8], int lanes, int lane, int& idx) {
  int o = lanes >> 1;
  bool up = (lane & o) != 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double send = up ? v[i] : v[i + 4];
    const double keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
  idx = up ? 4 : 0;
  o >>= 1;
  up = (lane & o) != 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double send = up ? v[i] : v[i + 2];
    const double keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
  idx += up ? 2 : 0;
  o >>= 1;
  up = (lane & o) != 0;
  {
    const double send = up ? v[0] : v[1];
    const double keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
  idx += up ? 1 : 0;
  for (o >>= 1; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}

struct Shared64 {
  uint32_t lg[256];                              // thread-part of the local index -> global bits
  double red[2][kThreads / 32][kMaxStepSlots];   // per-warp gradient sums of a step (double-buffered)
  int32_t slot[2][kMaxStepSlots];
  double dred[kThreads / 32];
  uint32_t gmap[16];
  uint32_t grp[4][4];
};

}  // namespace

// One complex128 pass: CTA c owns tiles c * tiles_per_cta .. (tile = sample *
// tiles_per_sample + tile within the sample); 2^(K-4) threads per tile, 16
// amplitudes per thread per step.
template <bool BWD, bool ROUNDS, bool RX = false>
__global__ void __launch_bounds__(kThreads, 1) pass64_kernel(const PassArgs64 a) {
  extern __shared__ __align__(16) double2 smem64[];
  __shared__ Shared64 sh;
  const PassDesc& pd = a.pd;
  const int K = pd.K;
  const int tl2 = K - kRegBits;
  const int Tt = 1 << tl2;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tiles_per_cta = kThreads >> tl2;
  const int64_t first_tile = (int64_t)blockIdx.x * tiles_per_cta;
  const int tile_in_cta = tid >> tl2;
  const uint32_t tau = (uint32_t)(tid & (Tt - 1));
  const int64_t total_tiles = (int64_t)a.B << a.tps_log2;
  const int64_t tile = first_tile + tile_in_cta;
  const bool active = tile < total_tiles;
  const int64_t b = active ? (tile >> a.tps_log2) : 0;
  const uint32_t t_in = active ? (uint32_t)(tile & ((1ll << a.tps_log2) - 1)) : 0u;
  const uint32_t outer = pdep(t_in, pd.outer_mask);
  const int64_t sbase = b << a.n_eff;
  double2* tp = smem64 + (tile_in_cta << K);
  double2* tl = smem64 + kTileAmps + (tile_in_cta << K);
  const int wpt = Tt >= 32 ? Tt / 32 : 1;  // warps per tile
  const int lanes = Tt < 32 ? Tt : 32;     // lanes per tile within a warp

  if (tid < 16) {
    sh.gmap[tid] = pd.gmap[tid];
    sh.grp[tid >> 2][tid & 3] = pd.groups[tid >> 2][tid & 3];
  }
  __syncthreads();
  for (int h = tid; h < Tt; h += kThreads) {
    uint32_t g = 0;
    for (int j = 0; j < tl2; ++j)
      if ((h >> j) & 1) g |= 1u << sh.gmap[kRegBits + j];
    sh.lg[h] = g;
  }
  __syncthreads();

  auto gidx = [&](uint32_t i) -> uint32_t { return outer | (i & 15u) | sh.lg[i >> 4]; };
  auto state_ptr = [&](int32_t code) -> double2* {
    if (code >= 0) return a.slots + (int64_t)code * a.slot_stride + sbase;
    return a.work + sbase;
  };

  // ---- bring psi (and lambda) in: local index i = it * Tt + tau -------------
  const int32_t psrc = pd.psi_src;
  if (psrc == SRC_GENERATE && a.psi_in) {
    // given initial states [B][2^n_in]; padding qubits (n_in <= bit < n_eff) are |0>
    const int64_t din = 1ll << a.n_in;
    const double2* src = a.psi_in + b * din;
#pragma unroll 4
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      const uint32_t g = gidx(i);
      const double2 v = (int64_t)g < din ? __ldcg(src + g) : make_double2(0.0, 0.0);
      if (active) tp[swz64(i)] = v;
    }
  } else if (psrc == SRC_GENERATE) {
    // psi_0 = (x) RY(x_q)|0>: a_x = prod_q (bit q of x ? sin(x_q/2) : cos(x_q/2))
    const double2* e = a.enc + b * a.n_eff;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      const uint32_t g = gidx(i);
      double pr = 1.0;
      for (int q = 0; q < a.n_eff; ++q) {
        const double2 f = __ldg(e + q);
        pr *= ((g >> q) & 1u) ? f.y : f.x;
      }
      if (active) tp[swz64(i)] = make_double2(pr, 0.0);
    }
  } else if (active) {
    // eight loads of each state in flight before their stores
    const bool half = (pd.flags & PF_SRC_H) != 0;
    const bool two = BWD && pd.lam_src == LAM_BUF;
    const double2* src = half ? nullptr : state_ptr(psrc);
    const float2* fsrc = half ? a.fslots + (int64_t)psrc * a.slot_stride + sbase : nullptr;
    const double2* lsrc = a.lam + sbase;
#pragma unroll
    for (int i0 = 0; i0 < 16; i0 += 8) {
      double2 vp[8], vl[8];
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const uint32_t g = gidx((uint32_t)(i0 + it) * Tt + tau);
        if (half) {
          const float2 h = __ldcg(fsrc + g);
          vp[it] = make_double2((double)h.x, (double)h.y);
        } else {
          vp[it] = __ldcg(src + g);
        }
        if (two) vl[it] = __ldcg(lsrc + g);
      }
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const uint32_t i = (uint32_t)(i0 + it) * Tt + tau;
        tp[swz64(i)] = vp[it];
        if (two) tl[swz64(i)] = vl[it];
      }
    }
  }
  if (BWD && pd.lam_src == LAM_BUF && psrc == SRC_GENERATE && active) {
    const double2* src = a.lam + sbase;
#pragma unroll 4
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      tl[swz64(i)] = __ldcg(src + gidx(i));
    }
  }
  __syncthreads();
  if (BWD && pd.lam_src == LAM_SEED) {
    // lambda_M = 2 (dL/dE_b) O psi_M (Eq. 4); (O psi)_x = i^{#Y} (-1)^{|(x^xm)&zm|} psi_{x^xm}
    const double scale = active ? 2.0 * a.dLdE[b] : 0.0;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      const uint32_t ip = i ^ pd.xm_local;
      const double2 v = ipow(tp[swz64(ip)], a.y_count);
      const uint32_t sg = __popc(gidx(ip) & a.z_mask) & 1u;
      tl[swz64(i)] = make_double2(flipd(v.x, sg) * scale, flipd(v.y, sg) * scale);
    }
    __syncthreads();
  }

  // ---- step program --------------------------------------------------------
  int buf = 0;
  int32_t pc = pd.op_begin;
  const uint2* ops = a.ops;
#pragma unroll 1
  while (pc < pd.op_end) {
    const uint2 op = __ldg(ops + pc++);
    const uint32_t code = op.x & 15u;
    if (ROUNDS && code == OP_STEP) {
      // ---- round step: rounds op.y .. op.y + nr - 1 on register group g
      const int g = (op.x >> 4) & 3;
      const int nr = (op.x >> 8) & 0xffff;
      const uint32_t lb0 = sh.grp[g][0], lb1 = sh.grp[g][1], lb2 = sh.grp[g][2], lb3 = sh.grp[g][3];
      const uint32_t gm = (1u << lb0) | (1u << lb1) | (1u << lb2) | (1u << lb3);
      const uint32_t base = pdep(tau, ((1u << K) - 1u) & ~gm);
      const uint32_t pb = swz64(base);
      const uint32_t so[4] = {swz64(1u << lb0), swz64(1u << lb1), swz64(1u << lb2), swz64(1u << lb3)};
      const uint32_t gb = gidx(base);
      const uint32_t pos[4] = {sh.gmap[lb0], sh.gmap[lb1], sh.gmap[lb2], sh.gmap[lb3]};
      double2 r[16];
      double2 l[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        r[j] = tp[pb ^ reg_offset(j, so)];
        if (BWD) l[j] = tl[pb ^ reg_offset(j, so)];
      }
      uint32_t D = 0;
#pragma unroll 1
      for (int k = 0; k < nr; ++k) {
        const size_t rr = (size_t)op.y + k;
        const RoundPar64& v = a.rpar[rr];
        if (!BWD) {
          const uint4 lk = __ldg(a.rounds + rr * (kFwdRoundWords / 4) + 1);
          // the items' rotation terms (-1: absent) in words 12..15
          const uint4 ty = __ldg(a.rounds + rr * (kFwdRoundWords / 4) + 3);
          rot_fwd64<0>(r, v.rot[0], D & 1u, D, (int)ty.x >= 0, RX && (lk.z & 1u));
          rot_fwd64<1>(r, v.rot[1], (D >> 1) & 1u, D, (int)ty.y >= 0, RX && ((lk.z >> 1) & 1u));
          rot_fwd64<2>(r, v.rot[2], (D >> 2) & 1u, D, (int)ty.z >= 0, RX && ((lk.z >> 2) & 1u));
          rot_fwd64<3>(r, v.rot[3], (D >> 3) & 1u, D, (int)ty.w >= 0, RX && ((lk.z >> 3) & 1u));
          diag64(r, v.ph);
          chain64(lk.x, gb, pos, a.n_eff, D);
        } else {
          const uint4 lk = __ldg(a.rounds + rr * (kBwdRoundWords / 4) + 2);
          const uint4 ty = __ldg(a.rounds + rr * (kBwdRoundWords / 4) + 1);
          chain64(lk.x, gb, pos, a.n_eff, D);
          double gv[8];
          diag_bwd64(r, l, v.ph, gv);
          rot_bwd64<0>(r, l, v.rot[0], D & 1u, D, gv[4], (int)ty.x >= 0, RX && (lk.z & 1u));
          rot_bwd64<1>(r, l, v.rot[1], (D >> 1) & 1u, D, gv[5], (int)ty.y >= 0, RX && ((lk.z >> 1) & 1u));
          rot_bwd64<2>(r, l, v.rot[2], (D >> 2) & 1u, D, gv[6], (int)ty.z >= 0, RX && ((lk.z >> 2) & 1u));
          rot_bwd64<3>(r, l, v.rot[3], (D >> 3) & 1u, D, gv[7], (int)ty.w >= 0, RX && ((lk.z >> 3) & 1u));
          int idx;
          const double sum = butterfly8_64(gv, lanes, lane, idx);
          const bool owner = (lane & ((lanes >> 3) - 1)) == 0;
          const int32_t term = __ldg(reinterpret_cast<const int32_t*>(a.rounds + rr * (kBwdRoundWords / 4)) + idx);
          if (Tt >= 32) {
            if (owner) {
              sh.red[buf][warp][k * 8 + idx] = sum;
              if (warp == 0) sh.slot[buf][k * 8 + idx] = term;
            }
          } else if (owner && active && term >= 0) {
            a.g_part[tile * a.n_slots + term] = 0.5 * sum;
          }
        }
      }
      pending64<BWD>(D, r, l);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        tp[pb ^ reg_offset(j, so)] = r[j];
        if (BWD) tl[pb ^ reg_offset(j, so)] = l[j];
      }
      __syncthreads();
      if (BWD && Tt >= 32) {
        const int nk = nr * 8;
        for (int e = tid; e < tiles_per_cta * nk; e += kThreads) {
          const int tc = e / nk, kk = e - tc * nk;
          const int64_t t2 = first_tile + tc;
          const int32_t term = sh.slot[buf][kk];
          if (t2 < total_tiles && term >= 0) {
            double sum = 0.0;
            for (int w = 0; w < wpt; ++w) sum += sh.red[buf][tc * wpt + w][kk];
            a.g_part[t2 * a.n_slots + term] = 0.5 * sum;
          }
        }
        buf ^= 1;
      }
    } else if (!ROUNDS && code == OP_STEP) {
      const int g = (op.x >> 4) & 3;
      const int nops = (op.x >> 8) & 0xffff;
      const int nk = (int)op.y;
      const uint32_t lb0 = sh.grp[g][0], lb1 = sh.grp[g][1], lb2 = sh.grp[g][2], lb3 = sh.grp[g][3];
      const uint32_t gm = (1u << lb0) | (1u << lb1) | (1u << lb2) | (1u << lb3);
      const uint32_t base = pdep(tau, ((1u << K) - 1u) & ~gm);
      const uint32_t pb = swz64(base);
      const uint32_t so[4] = {swz64(1u << lb0), swz64(1u << lb1), swz64(1u << lb2), swz64(1u << lb3)};
      const uint32_t gb = gidx(base);
      const uint32_t go[4] = {1u << sh.gmap[lb0], 1u << sh.gmap[lb1], 1u << sh.gmap[lb2], 1u << sh.gmap[lb3]};
      double2 r[16];
      double2 l[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        r[j] = tp[pb ^ reg_offset(j, so)];
        if (BWD) l[j] = tl[pb ^ reg_offset(j, so)];
      }
#pragma unroll 1
      for (int k = 0; k < nops; ++k) {
        const uint2 o = __ldg(ops + pc++);
        const uint32_t oc = o.x & 15u;
        if (!BWD && oc == OP_U) {
          const double2* u = a.mats + 4 * (size_t)(o.x >> 8);
          const double2 u00 = __ldg(u), u01 = __ldg(u + 1), u10 = __ldg(u + 2), u11 = __ldg(u + 3);
          switch ((o.x >> 4) & 3u) {
            case 0: apply_u64<0>(r, u00, u01, u10, u11); break;
            case 1: apply_u64<1>(r, u00, u01, u10, u11); break;
            case 2: apply_u64<2>(r, u00, u01, u10, u11); break;
            default: apply_u64<3>(r, u00, u01, u10, u11); break;
          }
        } else if (BWD && oc == OP_G) {
          const uint32_t rr = (o.x >> 4) & 3u, kind = (o.x >> 6) & 3u, ks = (o.x >> 8) & 0xffu;
          const double2 csv = __ldg(a.cs + o.y);
          double acc;
          if (kind == G_RZ) acc = bwd_dispatch64<G_RZ>(rr, r, l, csv.x, csv.y);
          else if (kind == G_RY) acc = bwd_dispatch64<G_RY>(rr, r, l, csv.x, csv.y);
          else acc = bwd_dispatch64<G_RX>(rr, r, l, csv.x, csv.y);
          for (int off = 1; off < lanes; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
          if (Tt >= 32) {
            if (lane == 0) sh.red[buf][warp][ks] = acc;
            if (tid == 0) sh.slot[buf][ks] = (int32_t)o.y;
          } else if (active && (lane & (Tt - 1)) == 0) {
            a.g_part[tile * a.n_slots + o.y] = 0.5 * acc;
          }
        } else if (oc == OP_CNOT) {
          const bool creg = ((o.y >> 8) & 1u) != 0;
          const uint32_t cb = o.y & 0xffu;
          switch ((o.x >> 4) & 3u) {
            case 0: cnot64<0, BWD>(r, l, creg, cb, gb); break;
            case 1: cnot64<1, BWD>(r, l, creg, cb, gb); break;
            case 2: cnot64<2, BWD>(r, l, creg, cb, gb); break;
            default: cnot64<3, BWD>(r, l, creg, cb, gb); break;
          }
        } else if (oc == OP_CHAIN || oc == OP_CZ) {
          const uint32_t links = o.y, c0 = o.y & 0xffu, c1 = (o.y >> 8) & 0xffu;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const uint32_t x = gb | reg_offset(j, go);
            const uint32_t sg = oc == OP_CHAIN ? (__popc(x & (x >> 1) & links) & 1u) : ((x >> c0) & (x >> c1) & 1u);
            r[j].x = flipd(r[j].x, sg);
            r[j].y = flipd(r[j].y, sg);
            if (BWD) {
              l[j].x = flipd(l[j].x, sg);
              l[j].y = flipd(l[j].y, sg);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        tp[pb ^ reg_offset(j, so)] = r[j];
        if (BWD) tl[pb ^ reg_offset(j, so)] = l[j];
      }
      __syncthreads();
      if (BWD && Tt >= 32) {
        // per-tile sums of the step's terms in warp order (deterministic)
        for (int e = tid; e < tiles_per_cta * nk; e += kThreads) {
          const int tc = e / nk, kk = e - tc * nk;
          const int64_t t2 = first_tile + tc;
          if (t2 < total_tiles) {
            double sum = 0.0;
            for (int w = 0; w < wpt; ++w) sum += sh.red[buf][tc * wpt + w][kk];
            a.g_part[t2 * a.n_slots + sh.slot[buf][kk]] = 0.5 * sum;
          }
        }
        buf ^= 1;
      }
    } else if (code == OP_CKPT || code == OP_ANCHOR) {
      double2* sp = a.slots + (int64_t)op.y * a.slot_stride + sbase;
#pragma unroll 4
      for (int it = 0; it < 16; ++it) {
        const uint32_t i = (uint32_t)it * Tt + tau;
        if (!active) continue;
        if (code == OP_CKPT) sp[gidx(i)] = tp[swz64(i)];
        else tp[swz64(i)] = sp[gidx(i)];
      }
      __syncthreads();
    }
  }

  // ---- write back ------------------------------------------------------------
  if (pd.psi_dst != BUF_NONE && (pd.flags & PF_DST_H)) {
    // memory-saving mode (Sec. 3.2): the stored pass output is rounded to complex64
    float2* dst = a.fslots + (int64_t)pd.psi_dst * a.slot_stride + sbase;
#pragma unroll 4
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      const double2 v = tp[swz64(i)];
      if (active) dst[gidx(i)] = make_float2((float)v.x, (float)v.y);
    }
  } else if (pd.psi_dst != BUF_NONE) {
    double2* dst = state_ptr(pd.psi_dst);
#pragma unroll 4
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      if (active) dst[gidx(i)] = tp[swz64(i)];
    }
  }
  if (BWD && pd.lam_dst == LAM_BUF) {
    double2* dst = a.lam + sbase;
#pragma unroll 4
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      if (active) dst[gidx(i)] = tl[swz64(i)];
    }
  }
  if (!BWD && (pd.flags & PF_EXPECT)) {
    // <psi|O|psi> partial of this tile (Eq. 1, matrix-free as in Appendix B.2)
    double acc = 0.0;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      const uint32_t ip = i ^ pd.xm_local;
      const double2 v = tp[swz64(i)];
      const double2 w = ipow(tp[swz64(ip)], a.y_count);
      const uint32_t sg = __popc(gidx(ip) & a.z_mask) & 1u;
      acc += flipd(v.x * w.x + v.y * w.y, sg);  // Re(conj(v) w) with the Z signs
    }
    for (int off = 1; off < lanes; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (Tt >= 32) {
      if (lane == 0) sh.dred[warp] = acc;
      __syncthreads();
      if (tid < tiles_per_cta) {
        const int64_t t2 = first_tile + tid;
        if (t2 < total_tiles) {
          double sum = 0.0;
          for (int w = 0; w < wpt; ++w) sum += sh.dred[tid * wpt + w];
          a.e_part[t2] = sum;
        }
      }
    } else if (active && (lane & (Tt - 1)) == 0) {
      a.e_part[tile] = acc;
    }
  }
}

// ---- observables whose X/Y qubits lie outside the tile (App. B.2) -------------
// CTA (b, t) sums Re(conj(a_x) (O a)_x) over x in [t * chunk, (t + 1) * chunk)
// of sample b; one float64 partial per CTA in the [B][rows] layout of the passes.
__global__ void __launch_bounds__(kThreads) expect_full64_kernel(const double2* psi, int n_eff, int64_t rows,
                                                                 uint32_t xm, uint32_t zm, uint32_t yc,
                                                                 double* e_part) {
  __shared__ double red[kThreads / 32];
  const int64_t dim = 1ll << n_eff;
  const int64_t chunk = dim / rows;
  const int64_t b = blockIdx.x / rows, t = blockIdx.x - b * rows;
  const double2* s = psi + b * dim;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < chunk; k += kThreads) {
    const uint32_t x = (uint32_t)(t * chunk + k), xp = x ^ xm;
    const double2 v = s[x];
    const double2 w = ipow(s[xp], yc);
    acc += flipd(v.x * w.x + v.y * w.y, __popc(xp & zm) & 1u);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) sum += red[w];
    e_part[blockIdx.x] = sum;
  }
}

// Adjoint seed lambda_x = 2 (dL/dE_b) (O psi_M)_x (Eq. 4) for every amplitude.
__global__ void seed_full64_kernel(const double2* psi, double2* lam, int n_eff, int64_t B, uint32_t xm,
                                   uint32_t zm, uint32_t yc, const double* dLdE) {
  const int64_t dim = 1ll << n_eff;
  const int64_t total = B * dim;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i >> n_eff;
    const uint32_t x = (uint32_t)(i & (dim - 1)), xp = x ^ xm;
    const double scale = 2.0 * dLdE[b];
    const double2 v = ipow(psi[b * dim + xp], yc);
    const uint32_t sg = __popc(xp & zm) & 1u;
    lam[i] = make_double2(flipd(v.x, sg) * scale, flipd(v.y, sg) * scale);
  }
}

// ---- launchers -------------------------------------------------------------------
cudaError_t launch_pass64(bool bwd, const PassArgs64& a, cudaStream_t st) {
  if (a.pd.K < kRegBits || a.pd.K > kMaxTileBits) return cudaErrorInvalidValue;
  const int tiles_per_cta = kThreads >> (a.pd.K - kRegBits);
  const int64_t total_tiles = (int64_t)a.B << a.tps_log2;
  const int64_t grid = (total_tiles + tiles_per_cta - 1) / tiles_per_cta;
  if (grid == 0) return cudaSuccess;
  const size_t smem = (size_t)(bwd ? 2 : 1) * kTileAmps * sizeof(double2);
  const bool rounds = a.rounds != nullptr, rx = rounds && a.rx_items;
  if (rounds && (a.rpar == nullptr || a.pd.K < 7)) return cudaErrorInvalidValue;  // 8 lanes per tile at least
  static OptIn once[6];
  const void* fn = bwd ? (rx       ? reinterpret_cast<const void*>(pass64_kernel<true, true, true>)
                          : rounds ? reinterpret_cast<const void*>(pass64_kernel<true, true>)
                                   : reinterpret_cast<const void*>(pass64_kernel<true, false>))
                       : (rx       ? reinterpret_cast<const void*>(pass64_kernel<false, true, true>)
                          : rounds ? reinterpret_cast<const void*>(pass64_kernel<false, true>)
                                   : reinterpret_cast<const void*>(pass64_kernel<false, false>));
  cudaError_t e = opt_in(fn, smem, once[(bwd ? 3 : 0) + (rx ? 2 : rounds ? 1 : 0)]);
  if (e != cudaSuccess) return e;
  if (bwd && rx) pass64_kernel<true, true, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
  else if (bwd && rounds) pass64_kernel<true, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
  else if (bwd) pass64_kernel<true, false><<<(unsigned)grid, kThreads, smem, st>>>(a);
  else if (rx) pass64_kernel<false, true, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
  else if (rounds) pass64_kernel<false, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
  else pass64_kernel<false, false><<<(unsigned)grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_expect_full64(const double2* psi, int n_eff, int64_t B, int64_t rows, uint32_t xm, uint32_t zm,
                                 uint32_t yc, double* e_part, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  expect_full64_kernel<<<(unsigned)(B * rows), kThreads, 0, st>>>(psi, n_eff, rows, xm, zm, yc, e_part);
  return cudaGetLastError();
}

cudaError_t launch_seed_full64(const double2* psi, double2* lam, int n_eff, int64_t B, uint32_t xm, uint32_t zm,
                               uint32_t yc, const double* dLdE, cudaStream_t st) {
  const int64_t total = B << n_eff;
  if (total == 0) return cudaSuccess;
  const int64_t want = (total + kThreads - 1) / kThreads;
  const unsigned grid = (unsigned)stream_grid(want);
  seed_full64_kernel<<<grid, kThreads, 0, st>>>(psi, lam, n_eff, B, xm, zm, yc, dLdE);
  return cudaGetLastError();
}

}  // namespace qf
