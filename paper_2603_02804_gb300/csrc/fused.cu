// Fused forward / adjoint pass kernels for sm_103a.
//
// One CTA (256 threads) owns 4096 amplitudes of shared memory per state:
// one tile of K = 12 tile bits, or 2^(12-K) tiles of a smaller circuit. A
// pass loads its tiles from HBM once (or generates psi_0 in place), runs the
// pass's step program on them in shared memory and registers, and stores them
// once: the forward and backward gate fusion of Secs. 3.2-3.3.
//
// Shared-memory layout: amplitude with local index i lives at i ^ ((i>>4)&15)
// (XOR swizzle on 8-byte words). Register groups are local nibbles, so the 16
// lanes of a half-warp always hit 16 distinct bank pairs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "kernels.h"

namespace qf {

// Sticky device error word (1: a bounded wait gave up); read and cleared by
// qf_device_status.
__device__ int g_qf_device_status = 0;

namespace {

__device__ __forceinline__ uint32_t swz(uint32_t i) { return i ^ ((i >> 4) & 15u); }

// Scatter the low bits of src into the set bits of mask (ascending).
__device__ __forceinline__ uint32_t pdep32(uint32_t src, uint32_t mask) {
  uint32_t r = 0;
  for (uint32_t bb = 1; mask; bb <<= 1) {
    const uint32_t low = mask & (0u - mask);
    if (src & bb) r |= low;
    mask ^= low;
  }
  return r;
}

__device__ __forceinline__ float flip(float v, uint32_t s) {
  return __int_as_float(__float_as_int(v) ^ (int)(s << 31));
}

// Pair (i, i+1), i even, to/from the swizzled tile.
__device__ __forceinline__ void st_pair(float2* sm, uint32_t i, float4 v) {
  const uint32_t p = swz(i);
  if (p & 1u) *reinterpret_cast<float4*>(sm + (p ^ 1u)) = make_float4(v.z, v.w, v.x, v.y);
  else *reinterpret_cast<float4*>(sm + p) = v;
}
__device__ __forceinline__ float4 ld_pair(const float2* sm, uint32_t i) {
  const uint32_t p = swz(i);
  if (p & 1u) {
    const float4 v = *reinterpret_cast<const float4*>(sm + (p ^ 1u));
    return make_float4(v.z, v.w, v.x, v.y);
  }
  return *reinterpret_cast<const float4*>(sm + p);
}

// ---- forward: fused 2x2 on register bit R -----------------------------------
template <int R>
__device__ __forceinline__ void apply_u(float2 (&r)[16], const float4 m0, const float4 m1) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    const float2 x = r[j], y = r[j1];
    r[j].x = m0.x * x.x - m0.y * x.y + m0.z * y.x - m0.w * y.y;
    r[j].y = m0.x * x.y + m0.y * x.x + m0.z * y.y + m0.w * y.x;
    r[j1].x = m1.x * x.x - m1.y * x.y + m1.z * y.x - m1.w * y.y;
    r[j1].y = m1.x * x.y + m1.y * x.x + m1.z * y.y + m1.w * y.x;
  }
}

// ---- backward: un-apply one rotation to psi and lambda on register bit R and
// return sum over the thread's pairs of Im<lambda|P|psi> taken before the
// un-apply. With du/dt = -(i/2) P u (Sec. 3.3), Re<lambda_j|du|psi_{j-1}> =
// (1/2) Im<lambda_j|P|psi_j>; the 1/2 is applied in float64 at the flush.
template <int R, int KIND>
__device__ __forceinline__ float bwd_gate(float2 (&p)[16], float2 (&l)[16], const float c,
                                          const float s) {
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    const float2 p0 = p[j], p1 = p[j1], l0 = l[j], l1 = l[j1];
    if (KIND == G_RZ) {
      acc += l0.x * p0.y - l0.y * p0.x - l1.x * p1.y + l1.y * p1.x;
      // u^dagger = diag(c + i s, c - i s)
      p[j] = make_float2(c * p0.x - s * p0.y, c * p0.y + s * p0.x);
      p[j1] = make_float2(c * p1.x + s * p1.y, c * p1.y - s * p1.x);
      l[j] = make_float2(c * l0.x - s * l0.y, c * l0.y + s * l0.x);
      l[j1] = make_float2(c * l1.x + s * l1.y, c * l1.y - s * l1.x);
    } else if (KIND == G_RY) {
      acc += l1.x * p0.x + l1.y * p0.y - l0.x * p1.x - l0.y * p1.y;
      // u^dagger = [[c, s], [-s, c]]
      p[j] = make_float2(c * p0.x + s * p1.x, c * p0.y + s * p1.y);
      p[j1] = make_float2(c * p1.x - s * p0.x, c * p1.y - s * p0.y);
      l[j] = make_float2(c * l0.x + s * l1.x, c * l0.y + s * l1.y);
      l[j1] = make_float2(c * l1.x - s * l0.x, c * l1.y - s * l0.y);
    } else {  // RX
      acc += l0.x * p1.y - l0.y * p1.x + l1.x * p0.y - l1.y * p0.x;
      // u^dagger = [[c, i s], [i s, c]]
      p[j] = make_float2(c * p0.x - s * p1.y, c * p0.y + s * p1.x);
      p[j1] = make_float2(c * p1.x - s * p0.y, c * p1.y + s * p0.x);
      l[j] = make_float2(c * l0.x - s * l1.y, c * l0.y + s * l1.x);
      l[j1] = make_float2(c * l1.x - s * l0.y, c * l1.y + s * l0.x);
    }
  }
  return acc;
}

template <int KIND>
__device__ __forceinline__ float bwd_dispatch_r(uint32_t r, float2 (&p)[16], float2 (&l)[16], float c,
                                                float s) {
  switch (r) {
    case 0: return bwd_gate<0, KIND>(p, l, c, s);
    case 1: return bwd_gate<1, KIND>(p, l, c, s);
    case 2: return bwd_gate<2, KIND>(p, l, c, s);
    default: return bwd_gate<3, KIND>(p, l, c, s);
  }
}

// CNOT with its target on register bit RT: swap the target pairs whose
// control is 1 (control: register bit cb when creg, else bit cb of the
// thread's base index gb). Self-inverse, so the adjoint applies the same.
template <int RT, bool BWD>
__device__ __forceinline__ void cnot_regs(float2 (&r)[16], float2 (&l)[16], bool creg, uint32_t cb, uint32_t gb) {
  const uint32_t cg = (gb >> cb) & 1u;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << RT)) continue;
    const int j1 = j | (1 << RT);
    const bool on = creg ? (((uint32_t)j >> cb) & 1u) != 0 : cg != 0;
    const float2 a = r[j], b = r[j1];
    r[j] = on ? b : a;
    r[j1] = on ? a : b;
    if (BWD) {
      const float2 c = l[j], d = l[j1];
      l[j] = on ? d : c;
      l[j1] = on ? c : d;
    }
  }
}

__device__ __forceinline__ uint32_t reg_off(uint32_t j, const uint32_t (&o)[4]) {
  return ((j & 1u) ? o[0] : 0u) ^ ((j & 2u) ? o[1] : 0u) ^ ((j & 4u) ? o[2] : 0u) ^
         ((j & 8u) ? o[3] : 0u);
}

// phase i^k times v
__device__ __forceinline__ float2 mul_ipow(float2 v, uint32_t k) {
  switch (k & 3u) {
    case 0: return v;
    case 1: return make_float2(-v.y, v.x);
    case 2: return make_float2(-v.x, -v.y);
    default: return make_float2(v.y, -v.x);
  }
}

// ---- round programs: pending CZ signs ------------------------------------------
// A thread's 16 registers hold psi~ with psi = D psi~, where D = (-1)^(c0 +
// sum_r A_r j_r) is the part of the CZ signs that is constant or linear in the
// register index j (bit 4 of D: c0, bits 0..3: A). D commutes with every
// diagonal gate; a gate on register bit r only sees the factor Z_r^(A_r),
// which is folded into that gate. CZs between two register bits (quadratic in
// j, the same for every thread) are signs of the round's diagonal table.
//
// Links L of one round, thread base index gb (register bits zero), register
// bit positions p[r]: x = gb ^ y(j) with disjoint supports, so each link q
// contributes gb_q gb_{q+1} (constant), gb_{q} y_{q+1} or y_q gb_{q+1} (linear)
// or y_q y_{q+1} (between register bits).
// Link q couples qubit q with q+1 mod n (link n-1 is a ring's CZ(n-1, 0); it
// never joins two register bits), hence the n-bit rotations.
__device__ __forceinline__ void link_terms(uint32_t L, uint32_t gb, int n, uint32_t& t2, uint32_t& u) {
  const uint32_t nmask = n >= 32 ? ~0u : ((1u << n) - 1u);
  const uint32_t t1 = L & gb;
  t2 = L & (((gb >> 1) | ((gb & 1u) << (n - 1))) & nmask);
  u = (((t1 << 1) | (t1 >> (n - 1))) & nmask) ^ t2;
}

// The pending-sign update of one round's links, from per-step constants of
// the thread (rgb = gb rotated right by one qubit, lgb = left, g12 = gb &
// rgb): as rotation distributes over &, u = rotl(L) & lgb ^ L & rgb (the
// link_terms u), and the constant part is |L & g12|. When the register bits
// sit on consecutive qubits (contig), A is one shift of u.
__device__ __forceinline__ void chain_pending(uint32_t L, uint32_t rgb, uint32_t lgb, uint32_t g12, int n,
                                                const uint32_t (&p)[4], bool contig, uint32_t& D) {
  const uint32_t nmask = n >= 32 ? ~0u : ((1u << n) - 1u);
  const uint32_t u = ((((L << 1) | (L >> (n - 1))) & nmask) & lgb) ^ (L & rgb);
  const uint32_t A = contig ? (u >> p[0]) & 15u
                            : ((u >> p[0]) & 1u) | (((u >> p[1]) & 1u) << 1) | (((u >> p[2]) & 1u) << 2) |
                                  (((u >> p[3]) & 1u) << 3);
  D ^= A | ((__popc(L & g12) & 1u) << 4);
}

// Multiply the registers by D (end of a step).
template <bool BWD>
__device__ __forceinline__ void apply_pending(uint32_t D, float2 (&r)[16], float2 (&l)[16]) {
  uint32_t S = (D & 16u) ? 0xFFFFu : 0u;
  S ^= (D & 1u) ? 0xAAAAu : 0u;
  S ^= (D & 2u) ? 0xCCCCu : 0u;
  S ^= (D & 4u) ? 0xF0F0u : 0u;
  S ^= (D & 8u) ? 0xFF00u : 0u;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int f = (int)((S << (31 - j)) & 0x80000000u);
    r[j].x = __int_as_float(__float_as_int(r[j].x) ^ f);
    r[j].y = __int_as_float(__float_as_int(r[j].y) ^ f);
    if (BWD) {
      l[j].x = __int_as_float(__float_as_int(l[j].x) ^ f);
      l[j].y = __int_as_float(__float_as_int(l[j].y) ^ f);
    }
  }
}

// RX(w) applied on register bit R: a rotation by -w/2 of the real pairs
// (re p0, im p1) and (re p1, im p0), three shears each (x += t y; y -= s x;
// x += t y). yq: the term's shear parameters (t, s, wrap parity) of the
// un-apply direction. A pending Z_R turns RX(w) into RX(-w).
template <int R>
__device__ __forceinline__ void rx_fwd(float2 (&r)[16], float4 yq, uint32_t a) {
  const int f = (int)(a << 31);
  const float t = __int_as_float(__float_as_int(yq.x) ^ f), s = __int_as_float(__float_as_int(yq.y) ^ f);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    float2 p0 = r[j], p1 = r[j1];
    p0.x = fmaf(t, p1.y, p0.x); p1.y = fmaf(-s, p0.x, p1.y); p0.x = fmaf(t, p1.y, p0.x);
    p1.x = fmaf(t, p0.y, p1.x); p0.y = fmaf(-s, p1.x, p0.y); p1.x = fmaf(t, p0.y, p1.x);
    r[j] = p0; r[j1] = p1;
  }
}

// The rotation of a forward item on register bit R (RY, or RX where rx; rx is
// uniform over the CTA): applying is the un-apply rotation the other way,
// (t, s) -> (-t, -s). A pending Z_R turns the rotation by w into one by -w.
// The rotation by w is u(phi) up to the sign (-1)^k of its wrap; prep folds
// the round's signs into the round's diagonal (a global sign of the state).
template <int R, bool RX>
__device__ __forceinline__ void rot_fwd(float2 (&r)[16], float4 yq, uint32_t a, uint32_t& D, bool rx) {
  if (RX && rx) {
    rx_fwd<R>(r, yq, a);
  } else {
    const int f = (int)(a << 31);
    const float tn = -__int_as_float(__float_as_int(yq.x) ^ f), sp = __int_as_float(__float_as_int(yq.y) ^ f);
    const float2 t2 = make_float2(tn, tn), ms2 = make_float2(sp, sp);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & (1 << R)) continue;
      const int j1 = j | (1 << R);
      float2 p0 = r[j], p1 = r[j1];
      // RY(w) on (p0, p1): rotation by +w/2 as three packed shears
      p0 = __ffma2_rn(t2, p1, p0);
      p1 = __ffma2_rn(ms2, p0, p1);
      p0 = __ffma2_rn(t2, p1, p0);
      r[j] = p0; r[j1] = p1;
    }
  }
}

// v *= (c + i s)
__device__ __forceinline__ void cmul(float2& v, float c, float s) {
  const float x = v.x;
  v.x = fmaf(c, x, -s * v.y);
  v.y = fmaf(s, x, c * v.y);
}

// The round's diagonal (its 4 RZ runs merged), applied: register amplitude j
// times the phase (cos, sin) held in ph[j / 2] (x, y for even j; z, w for odd
// j). An RZ run commutes with the rotations on the other register bits and
// with the pending signs, so the four run together, once per round, after the
// rotations (the adjoint un-applies them before its rotations, diag_bwd).
__device__ __forceinline__ void apply_diag(float2 (&r)[16], const float4* ph) {
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const float4 e = ph[m];
    cmul(r[2 * m], e.x, e.y);
    cmul(r[2 * m + 1], e.z, e.w);
  }
}

// Adjoint side of the round's diagonal: its RZ-run gradient terms, then the
// un-apply. g[r] = sum_j sigma_r(j) w_j with w_j = Im(conj(lambda_j) psi_j)
// and sigma_r(j) = +1 where bit r of j is clear, else -1 (the thread's share
// of Im<lambda|Z_r|psi>). w_j is unchanged by a diagonal acting on both states
// and Z_r commutes with the rotations on the other bits, so the four terms
// are taken together at the diagonal; the signed sums share partial sums (a
// Walsh transform along each register bit), and each pair of amplitudes is
// multiplied by its phases as it is read.
__device__ __forceinline__ void diag_bwd(float2 (&p)[16], float2 (&l)[16], const float4* ph, float (&g)[8]) {
  float s2[4];
  float d0 = 0.f, d1 = 0.f, se = 0.f;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const float4 e = ph[m];
    float2& p0 = p[2 * m];
    float2& p1 = p[2 * m + 1];
    float2& l0 = l[2 * m];
    float2& l1 = l[2 * m + 1];
    const float w0 = fmaf(l0.x, p0.y, -l0.y * p0.x);
    const float w1 = fmaf(l1.x, p1.y, -l1.y * p1.x);
    cmul(p0, e.x, e.y);
    cmul(l0, e.x, e.y);
    cmul(p1, e.z, e.w);
    cmul(l1, e.z, e.w);
    const float sm = w0 + w1;  // bit 0 summed out
    d0 += w0 - w1;
    if (m & 1) {
      s2[m >> 1] = se + sm;  // bits 0, 1 summed out
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

// Un-apply one rotation on register bit R by three shears and return the
// thread's sum of Im<lambda|P|psi> taken before it. A plane rotation by phi
// equals x += a y; y += b x; x += a y with a = -tan(phi/2), b = sin(phi)
// (exact; |a| <= 1 for |phi| <= pi/2), three FMAs per component; t =
// tan(w/4), s = sin(w/2).
//   RY: (x, y) <- RY(w)^dagger (x, y) = rotation by -w/2: a = t, b = -s.
template <int R, int KIND>
__device__ __forceinline__ float bwd_shear(float2 (&p)[16], float2 (&l)[16], const float t, const float s) {
  float acc = 0.f;
  float2 accp = make_float2(0.f, 0.f), accm = make_float2(0.f, 0.f);
  const float2 t2 = make_float2(t, t), ms2 = make_float2(-s, -s);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    const int j1 = j | (1 << R);
    float2 p0 = p[j], p1 = p[j1], l0 = l[j], l1 = l[j1];
    if (KIND == G_RX) {
      // Im<lambda|X|psi> per pair; RX(w)^dagger rotates (re p0, im p1) and
      // (re p1, im p0) by +w/2: x -= t y; y += s x; x -= t y
      acc += l0.x * p1.y - l0.y * p1.x + l1.x * p0.y - l1.y * p0.x;
      p0.x = fmaf(-t, p1.y, p0.x); p1.y = fmaf(s, p0.x, p1.y); p0.x = fmaf(-t, p1.y, p0.x);
      p1.x = fmaf(-t, p0.y, p1.x); p0.y = fmaf(s, p1.x, p0.y); p1.x = fmaf(-t, p0.y, p1.x);
      l0.x = fmaf(-t, l1.y, l0.x); l1.y = fmaf(s, l0.x, l1.y); l0.x = fmaf(-t, l1.y, l0.x);
      l1.x = fmaf(-t, l0.y, l1.x); l0.y = fmaf(s, l1.x, l0.y); l1.x = fmaf(-t, l0.y, l1.x);
    } else {
      // RY is real: the same shear acts on re and im, so each step is one
      // packed FFMA2 on the (re, im) pair; Im<lambda|Y|psi> per pair is
      // l1 . p0 - l0 . p1 (component-wise products, two packed accumulators).
      accp = __ffma2_rn(l1, p0, accp);
      accm = __ffma2_rn(l0, p1, accm);
      p0 = __ffma2_rn(t2, p1, p0);
      p1 = __ffma2_rn(ms2, p0, p1);
      p0 = __ffma2_rn(t2, p1, p0);
      l0 = __ffma2_rn(t2, l1, l0);
      l1 = __ffma2_rn(ms2, l0, l1);
      l0 = __ffma2_rn(t2, l1, l0);
    }
    p[j] = p0; p[j1] = p1; l[j] = l0; l[j1] = l1;
  }
  if (KIND == G_RY) acc = (accp.x + accp.y) - (accm.x + accm.y);
  return acc;
}

// The rotation of an adjoint item on register bit R (shear parameters (t, s);
// RX where rx, uniform over the CTA, else RY), un-applied after the round's
// diagonal; gy: its Im<lambda|P|psi>. With a pending Z_R the rotation
// un-applies as the one by +w (t, s negated) and gy changes sign. The wrap
// sign (u(phi) = -u(w) for odd k) is folded into the round's diagonal, which
// multiplies psi and lambda alike (their gradient terms do not change).
template <int R, bool RX = false>
__device__ __forceinline__ void rot_bwd(float2 (&p)[16], float2 (&l)[16], float4 yq, uint32_t a, uint32_t& D,
                                        float& gy, bool rx = false) {
  const int f = (int)(a << 31);
  const float t = __int_as_float(__float_as_int(yq.x) ^ f);
  const float s = __int_as_float(__float_as_int(yq.y) ^ f);
  const float g = RX && rx ? bwd_shear<R, G_RX>(p, l, t, s) : bwd_shear<R, G_RY>(p, l, t, s);
  gy = __int_as_float(__float_as_int(g) ^ f);
}

// Reduce 8 per-thread values over `lanes` lanes (8, 16 or 32; whole-warp
// call). Afterwards lane holds the lanes-sum of value *idx; the lanes with
// (lane & (lanes/8 - 1)) == 0 hold the 8 distinct values.
__device__ __forceinline__ float butterfly8(float (&v)[8], int lanes, int lane, int& idx) {
  int o = lanes >> 1;
  bool up = (lane & o) != 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = up ? v[i] : v[i + 4];
    const float keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
  idx = up ? 4 : 0;
  o >>= 1;
  up = (lane & o) != 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = up ? v[i] : v[i + 2];
    const float keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
  idx += up ? 2 : 0;
  o >>= 1;
  up = (lane & o) != 0;
  {
    const float send = up ? v[0] : v[1];
    const float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
  idx += up ? 1 : 0;
  for (o >>= 1; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}

// Two amplitudes as bfloat16 (re, im) pairs <-> float32 (round to nearest even).
__device__ __forceinline__ float4 bf16x4_to_f4(uint2 h) {
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ uint2 f4_to_bf16x4(float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  return make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}

// 16-byte asynchronous copy global -> shared (L2 only), and its fences.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Parameters of one round step, staged from the round-ordered tables: per
// round kRoundPar float4 (the items' rotation shears, then the round's
// diagonal) and the round record.
constexpr int kMaxRoundWords = kFwdRoundWords > kBwdRoundWords ? kFwdRoundWords : kBwdRoundWords;
struct StepPar {
  float4 v[kMaxStepRounds][kRoundPar];
  uint4 rec[kMaxStepRounds * (kMaxRoundWords / 4)];
};

// ---- tensor-core block path (tcgen05) --------------------------------------------
// A forward round applies u3 (x) u2 (x) u1 (x) u0 to the 16 amplitudes of a
// register group: a 16x16 complex block, i.e. a 32x32 real matrix on the
// (re, im) vector. A warpgroup's 128 columns (one per thread) form the MMA's
// M = 128 rows: D[m][n] = sum_k A[m][k] B[n][k], A = the columns' amplitudes
// (k < 16: re of amplitude k, else im of amplitude k - 16) in tensor memory,
// B = the round's real matrix (K-major, in shared memory), D in tensor memory.
// Split precision (3xTF32): A = Ah + Al, B = Bh + Bl with TF32 parts, and
// D = Ah Bh + Ah Bl + Al Bh accumulated in float32.
constexpr int kTcCols = 256;            // tensor-memory columns per CTA
constexpr int kTcWgCols = 96;           // per warpgroup: D, A hi, A lo (32 each)
constexpr int kTcBFloats = 2 * 1024;    // one round's B: hi then lo, 32x32 each
constexpr long long kTcSpinLimit = 1ll << 26;

// idesc for kind::tf32: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12 = 2),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory descriptor, K-major without swizzle: 8-row x 16-byte core
// matrices; LBO = 128 B between core matrices along K, SBO = 1024 B between
// 8-row groups; version 1 (bit 46).
__device__ __forceinline__ uint64_t tc_bdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cvt_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %3, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %4, p;\n}\n" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(acc), "r"(kTcIdesc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

// Wait for the mbarrier phase with the given parity; false after the spin limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t addr = smem_u32(mbar);
  for (long long it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

#define QF_R8(b) "%" #b "0, %" #b "1, %" #b "2, %" #b "3, %" #b "4, %" #b "5, %" #b "6, %" #b "7"

__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]),
        "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]),
        "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(u[k]);
}

// Per-CTA state of the tensor-core path.
struct TcCtx {
  uint32_t tmem;    // tensor-memory base (lane 0, first column)
  uint64_t* mbar;   // [2] one per warpgroup, in shared memory
  float* bsm;       // B staging: [2][kMaxStepRounds][kTcBFloats]
};

// Sign mask over the 16 register indices j of the round's CZ links (x = gb ^
// y(j)): constant part, parts linear in one register bit, and links between
// two register bits (bbits).
__device__ __forceinline__ uint32_t cz_mask16(uint32_t L, uint32_t bbits, uint32_t gb, const uint32_t (&p)[4], int n) {
  uint32_t t2, u;
  link_terms(L, gb, n, t2, u);
  uint32_t S = (__popc(t2 & gb) & 1u) ? 0xFFFFu : 0u;
  S ^= ((u >> p[0]) & 1u) ? 0xAAAAu : 0u;
  S ^= ((u >> p[1]) & 1u) ? 0xCCCCu : 0u;
  S ^= ((u >> p[2]) & 1u) ? 0xF0F0u : 0u;
  S ^= ((u >> p[3]) & 1u) ? 0xFF00u : 0u;
  S ^= (bbits & 1u) ? 0x8888u : 0u;
  S ^= (bbits & 2u) ? 0xC0C0u : 0u;
  S ^= (bbits & 4u) ? 0xF000u : 0u;
  return S;
}

// The rounds of one forward step on the tensor cores. r holds the thread's 16
// amplitudes (its column) on entry and exit. Warpgroup wg issues its own MMAs
// (M = its 128 columns) and waits on its own mbarrier; ph tracks the phase.
__device__ __forceinline__ void tc_rounds(const TcCtx& tc, const StepPar& P, int nr, const float* bst, uint32_t gb,
                                          const uint32_t (&pos)[4], int n, float2 (&r)[16], uint32_t& ph, int tid) {
  const int wg = tid >> 7, wq = (tid >> 5) & 3;
  const uint32_t col0 = tc.tmem + (uint32_t)(wg * kTcWgCols);
  const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
  const uint32_t d_col = col0, ah_col = col0 + 32, al_col = col0 + 64;
  float x[32];
  float n0 = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    x[j] = r[j].x;
    x[16 + j] = r[j].y;
    n0 = fmaf(x[j], x[j], fmaf(x[16 + j], x[16 + j], n0));
  }
#pragma unroll 1
  for (int k = 0; k < nr; ++k) {
    {
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        hi[q] = cvt_tf32(x[q]);
        lo[q] = cvt_tf32(x[q] - __uint_as_float(hi[q]));
      }
      tc_st32(ah_col | lane_off, hi);
      tc_st32(al_col | lane_off, lo);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    asm volatile("bar.sync %0, 128;" ::"r"(1 + wg) : "memory");
    if ((tid & 127) == 0) {
      tc_fence_after();
      const uint32_t bh = smem_u32(bst + (size_t)k * kTcBFloats), bl = bh + 4096u;
#pragma unroll
      for (int pr = 0; pr < 3; ++pr) {
        const uint32_t a = pr == 2 ? al_col : ah_col;
        const uint32_t b = pr == 1 ? bl : bh;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          tc_mma(d_col, a + 8u * kk, tc_bdesc(b + 256u * kk), (pr | kk) != 0 ? 1u : 0u);
      }
      tc_commit(tc.mbar + wg);
    }
    if (!mbar_wait(tc.mbar + wg, ph)) atomicExch(&g_qf_device_status, 1);
    ph ^= 1u;
    tc_fence_after();
    tc_ld32(d_col | lane_off, x);
    // CZ links after this round's rotations
    const uint4 lk = P.rec[k * (kFwdRoundWords / 4) + 1];
    const uint32_t S = cz_mask16(lk.x, lk.y, gb, pos, n);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int f = (int)((S << (31 - j)) & 0x80000000u);
      x[j] = __int_as_float(__float_as_int(x[j]) ^ f);
      x[16 + j] = __int_as_float(__float_as_int(x[16 + j]) ^ f);
    }
  }
  tc_fence_before();
  // The step acts on the column by a unitary (rotations and CZ signs), so its
  // norm is invariant; the tensor cores' float32 accumulation rounds toward
  // zero and shrinks it by a few ulp per round. Restore the norm.
  float n1 = 0.f;
#pragma unroll
  for (int q = 0; q < 32; ++q) n1 = fmaf(x[q], x[q], n1);
  const float sc = n1 > 0.f ? sqrtf(n0 / n1) : 1.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) r[j] = make_float2(x[j] * sc, x[16 + j] * sc);
}

}  // namespace

// ---------------------------------------------------------------------------
// Static shared memory of a pass (the tiles themselves are dynamic).
template <class Y>
__device__ void loss_block(int kind, double* E, const Y* y, int64_t B, double scale, double* loss, double* dLdE,
                           const double* e_part, int tps, int tid);

struct PassShared {
  StepPar par[2];
  uint32_t ticket;             // the CTA's finishing order (loss on the last CTA)
  uint32_t lg[256];
  uint32_t base[4][kThreads];  // per register group: the thread's tile index with the group's bits zero
  float red[2][kThreads / 32][kMaxStepSlots];
  int32_t slot[2][kMaxStepSlots];
  double dred[kThreads / 32];
  uint32_t gmap[16];
  uint32_t grp[4][4];
};

// One CTA's share of a pass: tiles first_tile .. first_tile + tiles_per_cta-1
// (tile = sample * tiles_per_sample + tile within the sample). Ends with a
// barrier, so a CTA may call it again for another pass or tile range. LOADS:
// tile loads in flight per thread and state (8 = the whole tile at once).
template <bool BWD, bool ROUNDS, int LOADS = 8, bool TC = false, bool RX = false>
__device__ __forceinline__ void pass_cta(const PassArgs& a, const int64_t first_tile, float2* smem, PassShared& sh,
                                         const TcCtx* tc = nullptr) {
  uint32_t (&s_lg)[256] = sh.lg;
  float (&s_red)[2][kThreads / 32][kMaxStepSlots] = sh.red;
  int32_t (&s_slot)[2][kMaxStepSlots] = sh.slot;
  double (&s_dred)[kThreads / 32] = sh.dred;
  uint32_t (&s_gmap)[16] = sh.gmap;
  uint32_t (&s_grp)[4][4] = sh.grp;

  const PassDesc& pd = a.pd;
  const int K = pd.K;
  const int tl2 = K - kRegBits;            // log2 threads per tile
  const int Tt = 1 << tl2;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tile_in_cta = tid >> tl2;
  const uint32_t tau = (uint32_t)(tid & (Tt - 1));
  const int tiles_per_cta = kThreads >> tl2;
  const int64_t total_tiles = (int64_t)a.B << a.tps_log2;
  const int64_t tile = first_tile + tile_in_cta;
  const bool active = tile < total_tiles;
  const int64_t b = active ? (tile >> a.tps_log2) : 0;
  const uint32_t t_in = active ? (uint32_t)(tile & ((1ll << a.tps_log2) - 1)) : 0u;
  const uint32_t outer = pdep32(t_in, pd.outer_mask);
  const int64_t dim = 1ll << a.n_eff;
  const int64_t sbase = b * dim;  // sample offset inside one state buffer
  float2* tp = smem + (tile_in_cta << K);
  float2* tl = smem + kTileAmps + (tile_in_cta << K);
  const int wpt = Tt >= 32 ? Tt / 32 : 1;  // warps per tile
  const int lanes = Tt < 32 ? Tt : 32;

  if (tid < 16) {
    s_gmap[tid] = pd.gmap[tid];
    s_grp[tid >> 2][tid & 3] = pd.groups[tid >> 2][tid & 3];
  }
  __syncthreads();
  for (int h = tid; h < (1 << tl2); h += kThreads) {
    uint32_t g = 0;
    for (int j = 0; j < tl2; ++j)
      if ((h >> j) & 1) g |= 1u << s_gmap[kRegBits + j];
    s_lg[h] = g;
  }
  __syncthreads();
  // each thread's base index per register group, once per pass (read back by
  // only the same thread, at every step of that group): computed while the
  // tile loads are in flight where the pass loads its tiles
  bool bases = false;
  auto set_bases = [&]() {
    for (int g = 0; g < 4; ++g) {
      // tau's bits scattered into the tile bits outside the group (pdep32 of
      // tau into the complement of the group's bits): a zero inserted at each
      // of the 4 group bits, lowest first, so that 4 steps replace K - 4
      uint32_t m = (1u << s_grp[g][0]) | (1u << s_grp[g][1]) | (1u << s_grp[g][2]) | (1u << s_grp[g][3]);
      uint32_t x = tau;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t low = m & (0u - m);
        const uint32_t hi = x & ~(low - 1u);
        x = (x ^ hi) | (hi << 1);
        m ^= low;
      }
      sh.base[g][tid] = x;
    }
    bases = true;
  };
  // (the persistent batch kernel and the RX instances keep the bases ahead
  // of the loads: their registers are tighter)
  constexpr bool kBasesInLoads = LOADS == 8 && !RX && !TC;
  if (!kBasesInLoads) set_bases();

  auto gidx = [&](uint32_t i) -> uint32_t { return outer | (i & 15u) | s_lg[i >> 4]; };
  auto state_ptr = [&](int32_t code) -> float2* {
    if (code >= 0) return a.slots + (int64_t)code * a.slot_stride + sbase;
    return a.work + sbase;
  };
  // (warp 0) the next round step at or after op q: its first round and count
  auto next_step = [&](int32_t q, uint32_t& rb, int& nr) -> bool {
    for (; q < pd.op_end; ++q) {
      const uint2 o = __ldg(a.ops + q);
      if ((o.x & 15u) == OP_STEP) {
        rb = o.y;
        nr = (int)((o.x >> 8) & 0xffffu);
        return true;
      }
    }
    return false;
  };
  // (tensor-core path, every thread) asynchronous copy of the B blocks of
  // rounds rb .. rb+nr-1 into staging buffer bb
  auto stage_b = [&](int bb, uint32_t rb, int nr) {
    const int n16 = nr * kTcBFloats / 4;
    const float* src = a.tcb + (size_t)rb * kTcBFloats;
    float* dst = tc->bsm + (size_t)bb * kMaxStepRounds * kTcBFloats;
    for (int e = tid; e < n16; e += kThreads) cp_async16(dst + 4 * e, src + 4 * e);
    cp_async_commit();
  };
  uint32_t ph = 0;  // tensor-core path: mbarrier phase of this thread's warpgroup
  // (warp 0) asynchronous copy of rounds rb .. rb+nr-1 into sh.par[pb]
  auto stage = [&](int pb, uint32_t rb, int nr) {
    constexpr int RW4 = (BWD ? kBwdRoundWords : kFwdRoundWords) / 4;
    const int nv = nr * kRoundPar, n_all = nv + nr * RW4;
    for (int e = lane; e < n_all; e += 32) {
      if (e < nv) cp_async16(&sh.par[pb].v[0][0] + e, a.rpar + (size_t)rb * kRoundPar + e);
      else cp_async16(&sh.par[pb].rec[e - nv], a.rounds + (size_t)rb * RW4 + (e - nv));
    }
    cp_async_commit();
  };

  // ---- bring psi (and lambda) in -------------------------------------------
  const int32_t psrc = pd.psi_src;
  if (psrc == SRC_GENERATE && a.psi_in) {
    // given initial states [B][2^n_in]; padding qubits (n_in <= bit < n_eff) are |0>
    const int64_t din = 1ll << a.n_in;
    const float2* src = a.psi_in + b * din;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const uint32_t i = 2u * ((uint32_t)it * Tt + tau);
      const uint32_t g = gidx(i);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (a.n_in == a.n_eff) {
        v = __ldcg(reinterpret_cast<const float4*>(src + g));
      } else if ((int64_t)g < din) {
        const float2 u0 = src[g], u1 = (int64_t)g + 1 < din ? src[g + 1] : make_float2(0.f, 0.f);
        v = make_float4(u0.x, u0.y, u1.x, u1.y);
      }
      if (active) st_pair(tp, i, v);
    }
  } else if (psrc == SRC_GENERATE) {
    // psi_0 = (x) RY(x_q)|0>: a_x = prod_q (bit q of x ? sin(x_q/2) : cos(x_q/2))
    const float2* e = a.enc + b * a.n_eff;
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
      const uint32_t i = 2u * ((uint32_t)it * Tt + tau);
      const uint32_t g = gidx(i);
      float pr = 1.f;
      for (int q = 1; q < a.n_eff; ++q) {
        const float2 f = __ldg(e + q);
        pr *= ((g >> q) & 1u) ? f.y : f.x;
      }
      const float2 f0 = __ldg(e);
      if (active) st_pair(tp, i, make_float4(pr * f0.x, 0.f, pr * f0.y, 0.f));
    }
  } else if (active) {
    // issue every load of the tile (psi, and lambda) before the first store
    const float2* src = state_ptr(psrc);
    const bool half = (pd.flags & PF_SRC_H) != 0;
    const __nv_bfloat162* hsrc =
        half ? reinterpret_cast<const __nv_bfloat162*>(a.hslots) + (int64_t)psrc * a.slot_stride + sbase : nullptr;
    const bool two = BWD && pd.lam_src == LAM_BUF;
    const float2* lsrc = a.lam + sbase;
#pragma unroll
    for (int i0 = 0; i0 < 8; i0 += LOADS) {
      float4 vp[LOADS], vl[LOADS];
#pragma unroll
      for (int it = 0; it < LOADS; ++it) {
        const uint32_t g = gidx(2u * ((uint32_t)(i0 + it) * Tt + tau));
        if (half) vp[it] = bf16x4_to_f4(__ldcg(reinterpret_cast<const uint2*>(hsrc + g)));
        else vp[it] = __ldcg(reinterpret_cast<const float4*>(src + g));
        if (two) vl[it] = __ldcg(reinterpret_cast<const float4*>(lsrc + g));
      }
      if (kBasesInLoads && i0 == 0) set_bases();
#pragma unroll
      for (int it = 0; it < LOADS; ++it) {
        const uint32_t i = 2u * ((uint32_t)(i0 + it) * Tt + tau);
        st_pair(tp, i, vp[it]);
        if (two) st_pair(tl, i, vl[it]);
      }
    }
  }
  if (!bases) set_bases();
  if (BWD && pd.lam_src == LAM_BUF && psrc == SRC_GENERATE && active) {
    const float2* src = a.lam + sbase;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const uint32_t i = 2u * ((uint32_t)it * Tt + tau);
      st_pair(tl, i, __ldcg(reinterpret_cast<const float4*>(src + gidx(i))));
    }
  }
  // round programs: stage the first step's parameters
  int sb = 0;
  if (ROUNDS && warp == 0) {
    uint32_t rb;
    int nr;
    if (next_step(pd.op_begin, rb, nr)) stage(0, rb, nr);
    cp_async_wait_all();
  }
  if (TC) {
    uint32_t rb;
    int nr;
    if (next_step(pd.op_begin, rb, nr)) stage_b(0, rb, nr);
    cp_async_wait_all();
    fence_proxy_async();  // B is read by the tensor cores (async proxy)
  }
  __syncthreads();
  if (BWD && pd.lam_src == LAM_SEED) {
    // lambda_M = 2 (dL/dE_b) O psi_M (Eq. 4); (O psi)_x = i^{#Y} (-1)^{|(x^xm)&zm|} psi_{x^xm}
    const float scale = active ? (float)(2.0 * a.dLdE[b]) : 0.f;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;  // single amplitudes here
      const uint32_t ip = i ^ pd.xm_local;
      const uint32_t gp = gidx(ip);
      float2 v = tp[swz(ip)];
      v = mul_ipow(v, a.y_count);
      const uint32_t sg = __popc(gp & a.z_mask) & 1u;
      tl[swz(i)] = make_float2(flip(v.x, sg) * scale, flip(v.y, sg) * scale);
    }
    __syncthreads();
  }

  // ---- step program ------------------------------------------------------------
  int buf = 0;
  int32_t pc = pd.op_begin;
  const uint2* ops = a.ops;
#pragma unroll 1
  while (pc < pd.op_end) {
    const uint2 op = __ldg(ops + pc++);
    const uint32_t code = op.x & 15u;
    if (ROUNDS && code == OP_STEP) {
      // ---- round step: straight-line rounds over the 4 register bits
      const int g = (op.x >> 4) & 3;
      const int nr = (op.x >> 8) & 0xffff;
      if (warp == 0) {
        // prefetch the next step's parameters while this one runs
        uint32_t rb;
        int nr2;
        if (next_step(pc, rb, nr2)) stage(sb ^ 1, rb, nr2);
      }
      if (TC) {
        uint32_t rb;
        int nr2;
        if (next_step(pc, rb, nr2)) stage_b(sb ^ 1, rb, nr2);
      }
      const StepPar& P = sh.par[sb];
      const uint32_t lb0 = s_grp[g][0], lb1 = s_grp[g][1], lb2 = s_grp[g][2], lb3 = s_grp[g][3];
      const uint32_t base = sh.base[g][tid];
      const uint32_t pb = swz(base);
      const uint32_t so[4] = {swz(1u << lb0), swz(1u << lb1), swz(1u << lb2), swz(1u << lb3)};
      const uint32_t gb = gidx(base);
      const uint32_t pos[4] = {s_gmap[lb0], s_gmap[lb1], s_gmap[lb2], s_gmap[lb3]};
      float2 r[16];
      float2 l[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        r[j] = tp[pb ^ reg_off(j, so)];
        if (BWD) l[j] = tl[pb ^ reg_off(j, so)];
      }
      const int nq = a.n_eff;
      const uint32_t nmask = nq >= 32 ? ~0u : ((1u << nq) - 1u);
      const uint32_t rgb = ((gb >> 1) | ((gb & 1u) << (nq - 1))) & nmask;
      const uint32_t lgb = ((gb << 1) | (gb >> (nq - 1))) & nmask;
      const uint32_t g12 = gb & rgb;
      const bool contig = pos[1] == pos[0] + 1 && pos[2] == pos[0] + 2 && pos[3] == pos[0] + 3;
      uint32_t D = 0;
      if constexpr (TC) {
        tc_rounds(*tc, P, nr, tc->bsm + (size_t)sb * kMaxStepRounds * kTcBFloats, gb, pos, a.n_eff, r, ph, tid);
      } else {
#pragma unroll 1
      for (int k = 0; k < nr; ++k) {
        if (!BWD) {
          const uint4 lk = P.rec[k * (kFwdRoundWords / 4) + 1];  // links, bbits, rx mask
          rot_fwd<0, RX>(r, P.v[k][0], D & 1u, D, lk.z & 1u);
          rot_fwd<1, RX>(r, P.v[k][1], (D >> 1) & 1u, D, (lk.z >> 1) & 1u);
          rot_fwd<2, RX>(r, P.v[k][2], (D >> 2) & 1u, D, (lk.z >> 2) & 1u);
          rot_fwd<3, RX>(r, P.v[k][3], (D >> 3) & 1u, D, (lk.z >> 3) & 1u);
          apply_diag(r, &P.v[k][4]);
          chain_pending(lk.x, rgb, lgb, g12, nq, pos, contig, D);
        } else {
          const uint4 lk = P.rec[k * (kBwdRoundWords / 4) + 2];  // links, bbits, rx mask
          chain_pending(lk.x, rgb, lgb, g12, nq, pos, contig, D);
          float v[8];
          diag_bwd(r, l, &P.v[k][4], v);
          rot_bwd<0, RX>(r, l, P.v[k][0], D & 1u, D, v[4], lk.z & 1u);
          rot_bwd<1, RX>(r, l, P.v[k][1], (D >> 1) & 1u, D, v[5], (lk.z >> 1) & 1u);
          rot_bwd<2, RX>(r, l, P.v[k][2], (D >> 2) & 1u, D, v[6], (lk.z >> 2) & 1u);
          rot_bwd<3, RX>(r, l, P.v[k][3], (D >> 3) & 1u, D, v[7], (lk.z >> 3) & 1u);
          int idx;
          float sum;
          bool owner;
          if (lanes == 32) {  // tiles of 9 qubits and more: the shuffle pattern as constants
            sum = butterfly8(v, 32, lane, idx);
            owner = (lane & 3) == 0;
          } else {
            sum = butterfly8(v, lanes, lane, idx);
            owner = (lane & ((lanes >> 3) - 1)) == 0;
          }
          const int32_t term =
              reinterpret_cast<const int32_t*>(&P.rec[k * (kBwdRoundWords / 4)])[idx];
          if (Tt >= 32) {
            if (owner) {
              s_red[buf][warp][k * 8 + idx] = sum;
              if (warp == 0) s_slot[buf][k * 8 + idx] = term;
            }
          } else if (owner && active && term >= 0) {
            a.g_part[tile * a.n_slots + term] = 0.5 * (double)sum;
          }
        }
      }
      apply_pending<BWD>(D, r, l);
      }  // CUDA-core rounds
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        tp[pb ^ reg_off(j, so)] = r[j];
        if (BWD) tl[pb ^ reg_off(j, so)] = l[j];
      }
      if (TC) {
        cp_async_wait_all();
        fence_proxy_async();
      } else if (warp == 0) {
        cp_async_wait_all();
      }
      __syncthreads();
      sb ^= 1;
      if (BWD && Tt >= 32 && a.g_accum) {
        // every tile of this call belongs to one sample: one thread per term sums
        // the tiles in order and adds to the sample's row (stored by its tile 0);
        // within a tile the warp sums add in float32, as the warp shuffles do,
        // then float64 across tiles
        const int nk = nr * 8;
        const int64_t b2 = first_tile >> a.tps_log2;
        const bool first = (first_tile & ((1ll << a.tps_log2) - 1)) == 0;
        for (int kk = kThreads - 1 - tid; kk < nk; kk += kThreads) {  // the last warp (warp 0 stages)
          const int32_t term = s_slot[buf][kk];
          if (term < 0) continue;
          double sum = 0.0;
          for (int tc = 0; tc < tiles_per_cta; ++tc)
            if (first_tile + tc < total_tiles) {
              float sf = 0.f;
              for (int w = 0; w < wpt; ++w) sf += s_red[buf][tc * wpt + w][kk];
              sum += (double)sf;
            }
          double* dst = a.g_part + b2 * a.n_slots + term;
          *dst = first ? 0.5 * sum : *dst + 0.5 * sum;
        }
        buf ^= 1;
      } else if (BWD && Tt >= 32) {
        // the tile's warp sums in float32 (one float64 value per tile and term)
        const int nk = nr * 8;
        for (int e = kThreads - 1 - tid; e < tiles_per_cta * nk; e += kThreads) {  // from the last warp
          const int tc = e / nk, kk = e - tc * nk;
          const int64_t t2 = first_tile + tc;
          const int32_t term = s_slot[buf][kk];
          if (t2 < total_tiles && term >= 0) {
            float sf = 0.f;
            for (int w = 0; w < wpt; ++w) sf += s_red[buf][tc * wpt + w][kk];
            a.g_part[t2 * a.n_slots + term] = (double)(0.5f * sf);
          }
        }
        buf ^= 1;
      }
    } else if (!ROUNDS && code == OP_STEP) {
      const int g = (op.x >> 4) & 3;
      const int nops = (op.x >> 8) & 0xffff;
      const int nk = (int)op.y;
      const uint32_t lb0 = s_grp[g][0], lb1 = s_grp[g][1], lb2 = s_grp[g][2], lb3 = s_grp[g][3];
      const uint32_t base = sh.base[g][tid];
      const uint32_t pb = swz(base);
      const uint32_t so[4] = {swz(1u << lb0), swz(1u << lb1), swz(1u << lb2), swz(1u << lb3)};
      const uint32_t gb = gidx(base);
      const uint32_t go[4] = {1u << s_gmap[lb0], 1u << s_gmap[lb1], 1u << s_gmap[lb2],
                              1u << s_gmap[lb3]};
      float2 r[16];
      float2 l[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        r[j] = tp[pb ^ reg_off(j, so)];
        if (BWD) l[j] = tl[pb ^ reg_off(j, so)];
      }
#pragma unroll 1
      for (int k = 0; k < nops; ++k) {
        const uint2 o = __ldg(ops + pc++);
        const uint32_t oc = o.x & 15u;
        if (!BWD && oc == OP_U) {
          const uint32_t m = o.x >> 8;
          const float4 m0 = __ldg(a.mats + 2 * m), m1 = __ldg(a.mats + 2 * m + 1);
          switch ((o.x >> 4) & 3u) {
            case 0: apply_u<0>(r, m0, m1); break;
            case 1: apply_u<1>(r, m0, m1); break;
            case 2: apply_u<2>(r, m0, m1); break;
            default: apply_u<3>(r, m0, m1); break;
          }
        } else if (BWD && oc == OP_G) {
          const uint32_t rr = (o.x >> 4) & 3u, kind = (o.x >> 6) & 3u, ks = (o.x >> 8) & 0xffu;
          const float2 csv = __ldg(a.cs + o.y);
          float acc;
          if (kind == G_RZ) acc = bwd_dispatch_r<G_RZ>(rr, r, l, csv.x, csv.y);
          else if (kind == G_RY) acc = bwd_dispatch_r<G_RY>(rr, r, l, csv.x, csv.y);
          else acc = bwd_dispatch_r<G_RX>(rr, r, l, csv.x, csv.y);
          for (int off = 1; off < lanes; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
          if (Tt >= 32) {
            if (lane == 0) s_red[buf][warp][ks] = acc;
            if (tid == 0) s_slot[buf][ks] = (int32_t)o.y;
          } else if (active && (lane & (Tt - 1)) == 0) {
            a.g_part[tile * a.n_slots + o.y] = 0.5 * (double)acc;
          }
        } else if (oc == OP_CNOT) {
          const bool creg = ((o.y >> 8) & 1u) != 0;
          const uint32_t cb = o.y & 0xffu;
          switch ((o.x >> 4) & 3u) {
            case 0: cnot_regs<0, BWD>(r, l, creg, cb, gb); break;
            case 1: cnot_regs<1, BWD>(r, l, creg, cb, gb); break;
            case 2: cnot_regs<2, BWD>(r, l, creg, cb, gb); break;
            default: cnot_regs<3, BWD>(r, l, creg, cb, gb); break;
          }
        } else if (oc == OP_CHAIN || oc == OP_CZ) {
          const uint32_t links = o.y, c0 = o.y & 0xffu, c1 = (o.y >> 8) & 0xffu;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const uint32_t x = gb | reg_off(j, go);
            const uint32_t sg = oc == OP_CHAIN ? (__popc(x & (x >> 1) & links) & 1u)
                                               : ((x >> c0) & (x >> c1) & 1u);
            r[j].x = flip(r[j].x, sg);
            r[j].y = flip(r[j].y, sg);
            if (BWD) {
              l[j].x = flip(l[j].x, sg);
              l[j].y = flip(l[j].y, sg);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        tp[pb ^ reg_off(j, so)] = r[j];
        if (BWD) tl[pb ^ reg_off(j, so)] = l[j];
      }
      __syncthreads();
      if (BWD && Tt >= 32) {
        for (int e = kThreads - 1 - tid; e < tiles_per_cta * nk; e += kThreads) {  // from the last warp
          const int tc = e / nk, kk = e - tc * nk;
          const int64_t t2 = first_tile + tc;
          if (t2 < total_tiles) {
            float sf = 0.f;
            for (int w = 0; w < wpt; ++w) sf += s_red[buf][tc * wpt + w][kk];
            a.g_part[t2 * a.n_slots + s_slot[buf][kk]] = (double)(0.5f * sf);
          }
        }
        buf ^= 1;
      }
    } else if (code == OP_CKPT || code == OP_ANCHOR) {
      float2* sp = a.slots + (int64_t)op.y * a.slot_stride + sbase;
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const uint32_t i = 2u * ((uint32_t)it * Tt + tau);
        if (!active) continue;
        if (code == OP_CKPT) *reinterpret_cast<float4*>(sp + gidx(i)) = ld_pair(tp, i);
        else st_pair(tp, i, *reinterpret_cast<const float4*>(sp + gidx(i)));
      }
      __syncthreads();
    }
  }

  // ---- write back -----------------------------------------------------------
  if (pd.psi_dst != BUF_NONE && (pd.flags & PF_DST_H)) {
    // memory-saving mode (Sec. 3.2): the stored copy is rounded to bfloat16
    __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(a.hslots) + (int64_t)pd.psi_dst * a.slot_stride + sbase;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const uint32_t i = 2u * ((uint32_t)it * Tt + tau);
      if (active) *reinterpret_cast<uint2*>(dst + gidx(i)) = f4_to_bf16x4(ld_pair(tp, i));
    }
  } else if (pd.psi_dst != BUF_NONE) {
    float2* dst = state_ptr(pd.psi_dst);
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const uint32_t i = 2u * ((uint32_t)it * Tt + tau);
      if (active) *reinterpret_cast<float4*>(dst + gidx(i)) = ld_pair(tp, i);
    }
  }
  if (BWD && pd.lam_dst == LAM_BUF) {
    float2* dst = a.lam + sbase;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const uint32_t i = 2u * ((uint32_t)it * Tt + tau);
      if (active) *reinterpret_cast<float4*>(dst + gidx(i)) = ld_pair(tl, i);
    }
  }
  if (!BWD && (pd.flags & PF_EXPECT)) {
    // <psi|O|psi> partial of this tile (Eq. 1, matrix-free as in Appendix B.2)
    float acc = 0.f;
#pragma unroll 1
    for (int it = 0; it < 16; ++it) {
      const uint32_t i = (uint32_t)it * Tt + tau;
      const uint32_t ip = i ^ pd.xm_local;
      const float2 v = tp[swz(i)];
      float2 w = mul_ipow(tp[swz(ip)], a.y_count);
      const uint32_t sg = __popc(gidx(ip) & a.z_mask) & 1u;
      acc += flip(v.x * w.x + v.y * w.y, sg);  // Re(conj(v) w) with the Z signs
    }
    double d = (double)acc;
    for (int off = 1; off < lanes; off <<= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (Tt >= 32) {
      if (lane == 0) s_dred[warp] = d;
      __syncthreads();
      if (tid < tiles_per_cta) {
        const int64_t t2 = first_tile + tid;
        if (t2 < total_tiles) {
          double sum = 0.0;
          for (int w = 0; w < wpt; ++w) sum += s_dred[tid * wpt + w];
          a.e_part[t2] = sum;
        }
      }
    } else if (active && (lane & (Tt - 1)) == 0) {
      a.e_part[tile] = d;
    }
  }
  __syncthreads();
  static_assert(kThreads == 256, "loss_block reduces over 256 threads");
  if (!BWD && a.done && (pd.flags & PF_EXPECT)) {
    // the last CTA to finish sums E over every CTA's partials and finishes
    // the loss (the partials are fenced before the count)
    __threadfence();
    __syncthreads();
    if (tid == 0) sh.ticket = atomicAdd(a.done, 1u);
    __syncthreads();
    if (sh.ticket == gridDim.x - 1) {
      __threadfence();
      loss_block<float>(a.loss_kind, a.E, a.y, a.B, a.loss_scale, a.loss, a.dLdE_out, a.e_part, 1 << a.tps_log2,
                        tid);
    }
    __syncthreads();
  }
}

// RX: round programs holding RX items (their own instance, so that programs
// of RZ / RY items keep the plain code). MINB: CTAs per SM the registers are
// budgeted for; a forward pass (one 32 KiB state per CTA) of more tiles than
// two CTAs per SM hold runs with three per SM.
template <bool BWD, bool ROUNDS, bool RX = false, int MINB = 2>
__global__ void __launch_bounds__(kThreads, MINB) pass_kernel(const PassArgs a) {
  extern __shared__ __align__(16) float2 smem[];
  __shared__ PassShared sh;
  pass_cta<BWD, ROUNDS, 8, false, RX>(a, (int64_t)blockIdx.x * (kThreads >> (a.pd.K - kRegBits)), smem, sh);
}

// Forward pass with the rounds on the tensor cores: one 12-qubit tile per
// CTA (two warpgroups of 128 columns). Dynamic shared memory: the tile, then
// two B staging buffers of kMaxStepRounds rounds.
__global__ void __launch_bounds__(kThreads, 2) tc_pass_kernel(const PassArgs a) {
  extern __shared__ __align__(16) float2 smem[];
  __shared__ PassShared sh;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int w = 0; w < 2; ++w)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[w])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  TcCtx ctx{tmem_slot, mbar, reinterpret_cast<float*>(smem + kTileAmps)};
  pass_cta<false, true, 8, true>(a, (int64_t)blockIdx.x, smem, sh, &ctx);
  // pass_cta ends with a barrier; every tensor-memory access is complete
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(kTcCols) : "memory");
}

// B blocks: element (n, k) of round r, n = output (re i | im i), k = input
// (re j | im j): U = u3 (x) u2 (x) u1 (x) u0 of the round's fused 2x2s,
// U[i][j] = prod_b u_b[i_b][j_b]; B[re i][re j] = Re U, B[re i][im j] = -Im U,
// B[im i][re j] = Im U, B[im i][im j] = Re U. Stored K-major (8-row x 16-byte
// core matrices, 128 B apart along K, 1024 B between row groups), TF32 hi at
// [0, 1024) and lo at [1024, 2048) of the round's block.
__global__ void tc_table_kernel(const uint4* fwd_rounds, int32_t n_rounds, const double* mats64, float* tcb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_rounds * 1024) return;
  const int64_t r = e >> 10;
  const int n = (int)((e >> 5) & 31), k = (int)(e & 31);
  const int i = n & 15, j = k & 15;
  const uint4 m = fwd_rounds[r * (kFwdRoundWords / 4)];
  const uint32_t mm[4] = {m.x, m.y, m.z, m.w};
  double re = 1.0, im = 0.0;
  for (int b = 0; b < 4; ++b) {
    const double* u = mats64 + 8 * (size_t)mm[b];
    const int ib = (i >> b) & 1, jb = (j >> b) & 1;
    const double ur = u[(ib * 2 + jb) * 2], ui = u[(ib * 2 + jb) * 2 + 1];
    const double t = re * ur - im * ui;
    im = re * ui + im * ur;
    re = t;
  }
  const bool ro = n < 16, ri = k < 16;
  const double v = ro ? (ri ? re : -im) : (ri ? im : re);
  const float vf = (float)v;
  const uint32_t hi = cvt_tf32(vf);
  const uint32_t lo = cvt_tf32((float)(v - (double)__uint_as_float(hi)));
  const int off = (n >> 3) * 256 + (k >> 2) * 32 + (n & 7) * 4 + (k & 3);
  tcb[r * kTcBFloats + off] = __uint_as_float(hi);
  tcb[r * kTcBFloats + 1024 + off] = __uint_as_float(lo);
}

// ---------------------------------------------------------------------------
// Gate tables from theta in float64, rounded once to float32 (or kept in
// float64 for complex128 plans): generic programs' fused 2x2 products
// (forward) and (cos, sin) of theta/2 per term (backward); round programs'
// per-round rotation shears and diagonal phases (both directions); (cos, sin)
// of x/2 per sample and qubit (encoding). Element 0 also clears the forward
// pass's CTA counter when a train step finishes its loss in that pass.
__device__ void prep_one(const PrepArgs& a, int64_t i);

__global__ void prep_kernel(const PrepArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && a.zero_word) *a.zero_word = 0u;
  prep_one(a, i);
}

namespace {

// One out-of-line float64 sincos shared by every table of prep, so that the
// kernel's element kinds run one copy of its code (prep runs after an L2
// flush in timed steps, and each inlined copy is fetched separately).
__device__ __noinline__ void sincos_prep(double x, double* s, double* c) { sincos(x, s, c); }

// Parameter p as float64 (float32 parameters are promoted exactly).
__device__ __forceinline__ double theta_at(const PrepArgs& a, int p) {
  return a.theta64 ? a.theta64[p] : (double)a.theta[p];
}

// Fused 2x2 product of fused entry m (float64, rounded once to float32).
__device__ void fused_u(const PrepArgs& a, int64_t m, float4& m0, float4& m1, double* u64 = nullptr) {
  double u[2][2][2] = {{{1, 0}, {0, 0}}, {{0, 0}, {1, 0}}};  // [row][col][re/im]
  for (int j = a.fuse_off[m]; j < a.fuse_off[m + 1]; ++j) {
    const FuseGate fg = a.fuse_gates[j];
    double s, c;
    sincos_prep(0.5 * (fg.param >= 0 ? theta_at(a, fg.param) : fg.angle), &s, &c);
    // g = c I - i s P
    double g[2][2][2];
    if (fg.kind == G_RX) {
      g[0][0][0] = c; g[0][0][1] = 0; g[0][1][0] = 0; g[0][1][1] = -s;
      g[1][0][0] = 0; g[1][0][1] = -s; g[1][1][0] = c; g[1][1][1] = 0;
    } else if (fg.kind == G_RY) {
      g[0][0][0] = c; g[0][0][1] = 0; g[0][1][0] = -s; g[0][1][1] = 0;
      g[1][0][0] = s; g[1][0][1] = 0; g[1][1][0] = c; g[1][1][1] = 0;
    } else {
      g[0][0][0] = c; g[0][0][1] = -s; g[0][1][0] = 0; g[0][1][1] = 0;
      g[1][0][0] = 0; g[1][0][1] = 0; g[1][1][0] = c; g[1][1][1] = s;
    }
    double t[2][2][2];
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 2; ++k) {
        double re = 0, im = 0;
        for (int q = 0; q < 2; ++q) {
          re += g[r][q][0] * u[q][k][0] - g[r][q][1] * u[q][k][1];
          im += g[r][q][0] * u[q][k][1] + g[r][q][1] * u[q][k][0];
        }
        t[r][k][0] = re;
        t[r][k][1] = im;
      }
    for (int r = 0; r < 2; ++r)
      for (int k = 0; k < 2; ++k) {
        u[r][k][0] = t[r][k][0];
        u[r][k][1] = t[r][k][1];
      }
  }
  m0 = make_float4((float)u[0][0][0], (float)u[0][0][1], (float)u[0][1][0], (float)u[0][1][1]);
  m1 = make_float4((float)u[1][0][0], (float)u[1][0][1], (float)u[1][1][0], (float)u[1][1][1]);
  if (u64)
    for (int q = 0; q < 8; ++q) u64[q] = u[q >> 2][(q >> 1) & 1][q & 1];
}

// A term's angle is the sum of its parameters (a merged run of RZ gates).
__device__ double term_angle(const PrepArgs& a, int64_t t) {
  double phi = a.term_const ? a.term_const[t] : 0.0;
  for (int j = a.term_off[t]; j < a.term_off[t + 1]; ++j) phi += theta_at(a, a.term_params[j]);
  return phi;
}

// term_angle of the terms t[0..3] (-1: none, angle 0) with the loads of the
// four terms issued together: the index ranges and constants, then the first
// two parameters of each, then their values (the same summation order as
// term_angle; a term of more than two parameters finishes in a loop).
__device__ void term_angles4(const PrepArgs& a, const int32_t* t, double (&phi)[4]) {
  int b0[4], b1[4], p0[4], p1[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const bool on = t[r] >= 0;
    b0[r] = on ? a.term_off[t[r]] : 0;
    b1[r] = on ? a.term_off[t[r] + 1] : 0;
    phi[r] = on && a.term_const ? a.term_const[t[r]] : 0.0;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    p0[r] = b1[r] > b0[r] ? a.term_params[b0[r]] : -1;
    p1[r] = b1[r] > b0[r] + 1 ? a.term_params[b0[r] + 1] : -1;
  }
  double v0[4], v1[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    v0[r] = p0[r] >= 0 ? theta_at(a, p0[r]) : 0.0;
    v1[r] = p1[r] >= 0 ? theta_at(a, p1[r]) : 0.0;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (p0[r] >= 0) phi[r] += v0[r];
    if (p1[r] >= 0) phi[r] += v1[r];
    for (int j = b0[r] + 2; j < b1[r]; ++j) phi[r] += theta_at(a, a.term_params[j]);
  }
}

// The angle of a resolved round term (the same summation order as
// term_angle: the constant, then the parameters).
__device__ __forceinline__ double round_term_angle(const PrepArgs& a, const RoundTerm& e) {
  if (e.p0 <= -2) return term_angle(a, -2 - e.p0);
  double phi = e.c;
  if (e.p0 >= 0) phi += theta_at(a, e.p0);
  if (e.p1 >= 0) phi += theta_at(a, e.p1);
  return phi;
}

// u(phi) = (-1)^k u(w) with w = phi - 2 pi k in [-pi, pi] (k the nearest
// integer to phi / 2 pi): the rotation by w/2 as three shears needs tan(w/4)
// (|.| <= 1) and sin(w/2); angle 0 (also a missing term) gives all zero.
// tan(w/4) = sin(w/2) / (1 + cos(w/2)) (the half-angle identity; the
// denominator lies in [1, 2] for |w/2| <= pi/2), so one float64 sincos gives
// both.
__device__ __forceinline__ double wrap_count(double phi) {
  return rint(phi * (1.0 / 6.283185307179586476925286766559));
}

__device__ void shear_params(double phi, double& tq, double& sh, int& parity) {
  const double two_pi = 6.283185307179586476925286766559;
  const double k = wrap_count(phi);
  const double w = phi - two_pi * k;
  double c;
  sincos_prep(0.5 * w, &sh, &c);
  tq = sh / (1.0 + c);
  parity = ((long long)k) & 1;
}

__device__ float4 shear_of(double phi) {
  double tq, sh;
  int parity;
  shear_params(phi, tq, sh, parity);
  return make_float4((float)tq, (float)sh, __int_as_float(parity), 0.f);
}

// The same in float64 (complex128 round programs).
__device__ Shear64 shear64_of(double phi) {
  Shear64 r{0.0, 0.0, 0, 0};
  int parity;
  shear_params(phi, r.t, r.s, parity);
  r.wrap = parity;
  return r;
}

// The diagonal of a round: its RZ runs (angles phi_r; 0 for a missing term)
// act on register index j as e^{-i a_j} with a_j = sum_r sigma_r(j) phi_r / 2,
// sigma_r(j) = +1 where bit r of j is clear, else -1 (RZ(phi) =
// diag(e^{-i phi/2}, e^{i phi/2})), and its CZ links between register bits r
// and r + 1 (bit r of bbits) as -1 where both bits of j are set. Gives
// (cos, sin) of the applied phase (forward: -a_j) or of the un-applied one
// (backward: +a_j) for j = m, and the CZ signs of m and its complement
// 15 - m: a_{15-m} = -a_m, so one float64 sincos of the summed angle serves both.
__device__ void diag_phase_pair(const double (&phi)[4], uint32_t bbits, int m, bool apply, double& c, double& s,
                                bool& f0, bool& f1) {
  double al = 0.0;
  for (int r = 0; r < 4; ++r) al += ((m >> r) & 1) ? -phi[r] : phi[r];
  al *= apply ? -0.5 : 0.5;
  sincos_prep(al, &s, &c);
  const int mc = 15 - m;
  f0 = __popc(bbits & (uint32_t)m & (uint32_t)(m >> 1)) & 1;
  f1 = __popc(bbits & (uint32_t)mc & (uint32_t)(mc >> 1)) & 1;
}

// neg: the round's items' wrap signs multiply to -1; the phases carry it.
__device__ void diag_phases(const double (&phi)[4], uint32_t bbits, int m, bool apply, bool neg, float2* ph) {
  double cd, sd;
  bool f0, f1;
  diag_phase_pair(phi, bbits, m, apply, cd, sd, f0, f1);
  const float c = neg ? -(float)cd : (float)cd, s = neg ? -(float)sd : (float)sd;
  ph[m] = f0 ? make_float2(-c, -s) : make_float2(c, s);
  ph[15 - m] = f1 ? make_float2(-c, s) : make_float2(c, -s);
}

// The same in float64 (complex128 round programs).
__device__ void diag_phases64(const double (&phi)[4], uint32_t bbits, int m, bool apply, double2* ph) {
  double c, s;
  bool f0, f1;
  diag_phase_pair(phi, bbits, m, apply, c, s, f0, f1);
  ph[m] = f0 ? make_double2(-c, -s) : make_double2(c, s);
  ph[15 - m] = f1 ? make_double2(-c, s) : make_double2(c, -s);
}

}  // namespace

// Element i of the tables: fused matrices, terms, encodings, then (round
// programs) the forward and backward round parameters in round order.
__device__ void prep_one(const PrepArgs& a, int64_t i) {
  if (i < a.n_fused) {
    float4 m0, m1;
    fused_u(a, i, m0, m1, a.mats64 ? a.mats64 + 8 * i : nullptr);
    if (a.mats) {
      a.mats[2 * i] = m0;
      a.mats[2 * i + 1] = m1;
    }
    return;
  }
  i -= a.n_fused;
  if (i < a.n_terms) {
    if (a.cs64) {
      double s, c;
      sincos_prep(0.5 * term_angle(a, i), &s, &c);
      a.cs64[i] = make_double2(c, s);
    } else {
      double s, c;
      sincos_prep(0.5 * term_angle(a, i), &s, &c);
      a.cs[i] = make_float2((float)c, (float)s);
    }
    return;
  }
  i -= a.n_terms;
  if (i < (int64_t)a.B * a.n_eff) {
    const int64_t bb = i / a.n_eff;
    const int q = (int)(i - bb * a.n_eff);
    double s = 0.0, c = 1.0;  // a padding qubit stays |0>
    if (q < a.n) {
      // simulated bit q holds circuit qubit (q - qshift) mod n
      const int qc = a.qshift ? (q + a.n - a.qshift) % a.n : q;
      sincos_prep(0.5 * (a.x64 ? a.x64[bb * a.n + qc] : (double)a.x[bb * a.n + qc]), &s, &c);
    }
    if (a.enc64) a.enc64[i] = make_double2(c, s);
    else a.enc[i] = make_float2((float)c, (float)s);
    return;
  }
  i -= (int64_t)a.B * a.n_eff;
  // per round the 4 rotation shears, then the merged diagonal (float32 tables,
  // or float64 ones for complex128 plans)
  bool fwd = i < (int64_t)kRoundPar * a.n_rpf;
  if (!fwd) i -= (int64_t)kRoundPar * a.n_rpf;
  if (!fwd && i >= (int64_t)kRoundPar * a.n_rpb) return;
  const int64_t r = i / kRoundPar;
  const int e = (int)(i - r * kRoundPar);
  const int32_t* rec = fwd ? reinterpret_cast<const int32_t*>(a.rpf_src) + r * kFwdRoundWords
                           : reinterpret_cast<const int32_t*>(a.rpb_src) + r * kBwdRoundWords;
  const int32_t* tz = fwd ? rec + 8 : rec;
  const int32_t* ty = fwd ? rec + 12 : rec + 4;
  // the round's terms resolved at plan time (their loads issue together), or
  // through the term maps
  const RoundTerm* rt = fwd ? a.rpf_terms : a.rpb_terms;
  if (rt) rt += r * 8;
  const bool f64 = a.rpf64 || a.rpb64;
  if (e < 4) {
    const double phi = rt ? round_term_angle(a, rt[e]) : (ty[e] >= 0 ? term_angle(a, ty[e]) : 0.0);
    if (f64) (fwd ? a.rpf64 : a.rpb64)[r].rot[e] = shear64_of(phi);
    else (fwd ? a.rpf : a.rpb)[r * kRoundPar + e] = shear_of(phi);
    return;
  }
  const uint32_t bbits = (uint32_t)(fwd ? rec[5] : rec[9]);
  double phi[4];
  if (rt) {
#pragma unroll
    for (int q = 0; q < 4; ++q) phi[q] = round_term_angle(a, rt[4 + q]);
  } else {
    term_angles4(a, tz, phi);
  }
  if (f64) {
    diag_phases64(phi, bbits, e - 4, fwd, (fwd ? a.rpf64 : a.rpb64)[r].ph);
  } else {
    // the product of the 4 rotations' wrap signs (-1)^k, the same k as their shears
    long long k = 0;
    for (int q = 0; q < 4; ++q) {
      const double phr = rt ? round_term_angle(a, rt[q]) : (ty[q] >= 0 ? term_angle(a, ty[q]) : 0.0);
      k += (long long)wrap_count(phr);
    }
    diag_phases(phi, bbits, e - 4, fwd, (k & 1) != 0,
                reinterpret_cast<float2*>((fwd ? a.rpf : a.rpb) + r * kRoundPar + 4));
  }
}

// E_b = sum over the tiles of sample b, in tile order (deterministic).
__global__ void e_reduce_kernel(const double* e_part, int64_t B, int tps, double* E) {
  const int64_t bb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bb >= B) return;
  double s = 0.0;
  for (int t = 0; t < tps; ++t) s += e_part[bb * tps + t];
  E[bb] = s;
}

// The same for many partials per sample: one block per sample, thread k sums
// partials k, k + 256, ... in order, then a fixed tree (bitwise repeatable).
__global__ void __launch_bounds__(256) e_reduce_block_kernel(const double* e_part, int tps, double* E) {
  __shared__ double red[256];
  const int64_t bb = blockIdx.x;
  double s = 0.0;
  for (int t = threadIdx.x; t < tps; t += 256) s += e_part[bb * tps + t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) E[bb] = red[0];
}

// Stage 1 of a two-stage gradient reduction over partials [row][slot]
// (slots contiguous): block (group g, chunk c) sums rows
// g * rows_per_group + c * kGReduceChunk .. (chunk end) of each slot in row
// order; consecutive threads read consecutive slots of a row.
__global__ void g_partial_kernel(const double* g_part, int64_t rows_per_group, int64_t chunks, int64_t slot_stride,
                                 int S, double* out) {
  const int64_t gc = blockIdx.x;
  const int64_t g = gc / chunks, c = gc - g * chunks;
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int64_t r0 = g * rows_per_group + c * kGReduceChunk;
  const int64_t r1 = g * rows_per_group + min(rows_per_group, (c + 1) * (int64_t)kGReduceChunk);
  double acc = 0.0;
  for (int64_t r = r0; r < r1; ++r) acc += g_part[r * slot_stride + s];
  out[gc * S + s] = acc;
}

// grad[p] (or grad[b][p]) = sum over tiles, then over the slots of p, in a
// fixed order.
__global__ void g_reduce_kernel(const GradReduceArgs a) {
  // one warp per output value; lane k sums rows k, k+32, ... and the warp
  // combines the 32 lane sums in a fixed butterfly (bitwise repeatable)
  const int64_t out = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t n_out = a.per_sample ? (int64_t)a.B * a.n_params : a.n_params;
  if (out >= n_out) return;  // whole warps exit together
  const int64_t bb = a.per_sample ? out / a.n_params : 0;
  const int p = (int)(a.per_sample ? out - bb * a.n_params : out);
  const int64_t rows = a.per_sample ? a.tps : (int64_t)a.B * a.tps;
  const int64_t row0 = a.per_sample ? bb * a.tps : 0;
  double s = 0.0;
  for (int k = a.param_off[p]; k < a.param_off[p + 1]; ++k) {
    const int64_t col = (int64_t)a.param_slots[k] * a.slot_step;
#pragma unroll 8
    for (int64_t t = lane; t < rows; t += 32) s += a.g_part[(row0 + t) * a.slot_stride + col];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) a.grad[out] = s;
}

// Loss and dL/dE in one block of 256 threads with a fixed-order reduction
// (warp shuffles, then the 8 warp sums in warp 0); labels float32, or float64
// for complex128 plans. scale = 2 / B (MSE: dL/dE_i = scale (E_i - y_i)).
// With e_part: E_i is first summed from its tps partials in tile order (as
// e_reduce_kernel does) and stored; they are read from L2, as they may come
// from other CTAs of the same launch.
template <class Y>
__device__ void loss_block(int kind, double* E, const Y* y, int64_t B, double scale, double* loss, double* dLdE,
                           const double* e_part, int tps, int tid) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = tid; i < B; i += 256) {
    double Ei;
    if (e_part) {
      Ei = 0.0;
      for (int t = 0; t < tps; ++t) Ei += __ldcg(e_part + i * tps + t);
      E[i] = Ei;
    } else {
      Ei = E[i];
    }
    if (kind == 1) {
      const double d = Ei - (double)y[i];
      s += d * d;
      dLdE[i] = scale * d;
    } else {
      s += Ei;
      dLdE[i] = 1.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid < 32) {
    s = tid < 8 ? red[tid] : 0.0;
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) loss[0] = kind == 1 ? s * (0.5 * scale) : s;
  }
}

template <class Y>
__global__ void __launch_bounds__(256) loss_kernel(int kind, double* E, const Y* y, int64_t B, double scale,
                                                   double* loss, double* dLdE, const double* e_part, int tps) {
  loss_block<Y>(kind, E, y, B, scale, loss, dLdE, e_part, tps, threadIdx.x);
}

// ---- batched persistent launch -------------------------------------------------
namespace {

template <class T>
__device__ __forceinline__ T* rebase(T* p, char* base) {
  return reinterpret_cast<T*>(base + reinterpret_cast<uintptr_t>(p));
}
template <class T>
__device__ __forceinline__ const T* rebase(const T* p, char* base) {
  return reinterpret_cast<const T*>(base + reinterpret_cast<uintptr_t>(p));
}

__device__ __forceinline__ int find_circuit(const int64_t* off, int n, int64_t i) {
  int lo = 0, hi = n;  // off[lo] <= i < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Copy a circuit's pass arguments into shared memory with pass descriptor pd
// and the workspace pointers rebased.
__device__ void load_args(PassArgs& dst, const PassArgs& src, const PassDesc& pd, char* ws) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(&src);
  uint32_t* d = reinterpret_cast<uint32_t*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(PassArgs) / 4); i += blockDim.x) d[i] = s[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    dst.pd = pd;
    dst.mats = rebase(dst.mats, ws);
    dst.rpar = rebase(dst.rpar, ws);
    dst.enc = rebase(dst.enc, ws);
    dst.work = rebase(dst.work, ws);
    dst.lam = rebase(dst.lam, ws);
    dst.slots = rebase(dst.slots, ws);
    dst.dLdE = rebase(dst.dLdE, ws);
    dst.e_part = rebase(dst.e_part, ws);
    dst.g_part = rebase(dst.g_part, ws);
  }
  __syncthreads();
}

__device__ void run_item_pass(bool bwd, const PassArgs& a, int32_t b0) {
  extern __shared__ __align__(16) float2 smem[];
  __shared__ PassShared sh;
  const int tpc = kThreads >> (a.pd.K - kRegBits);
  // tpc tiles per call: with one tile per sample (tps = 1) the item's samples
  // b0 .. b0 + tpc - 1 in one call, else the tiles of sample b0 in turn
  const int64_t tps = 1ll << a.tps_log2;
  for (int64_t t = 0; t < tps; t += tpc) {
    if (bwd) pass_cta<true, true, 2>(a, (int64_t)b0 * tps + t, smem, sh);
    else pass_cta<false, true, 2>(a, (int64_t)b0 * tps + t, smem, sh);
  }
}

}  // namespace

__global__ void batch_prep_kernel(const BatchArgs a, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int c = find_circuit(a.prep_off, a.n_circ, i);
  PrepArgs p = a.circ[c].prep;
  p.theta = a.theta + a.circ[c].theta_off;
  p.x = a.x + a.circ[c].x_off;
  p.mats = rebase(p.mats, a.ws);
  p.rpf = rebase(p.rpf, a.ws);
  p.rpb = rebase(p.rpb, a.ws);
  p.enc = rebase(p.enc, a.ws);
  prep_one(p, i - a.prep_off[c]);
}

// Persistent kernel: CTAs take work items (one sample, or a group of small
// samples, of one circuit; largest first) from an atomic queue and run the
// item's forward passes, its loss derivative and its adjoint passes
// themselves, so items never wait on each other.
__global__ void __launch_bounds__(kThreads, 2) batch_kernel(const BatchArgs a) {
  __shared__ PassArgs s_a;
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= a.n_items) return;
    const BatchItem item = a.items[it];
    const BatchCircuit& C = a.circ[item.c];
    for (int p = 0; p < C.n_fwd; ++p) {
      load_args(s_a, C.fa, C.fwd[p], a.ws);
      run_item_pass(false, s_a, item.b0);
    }
    // E and dL/dE of the item's samples (their tiles were written by this CTA)
    {
      const int64_t B = C.fa.B;
      const int64_t tps = 1ll << C.fa.tps_log2;
      const int ns = (int)min((int64_t)C.samples_per_item, B - item.b0);
      if ((int)threadIdx.x < ns) {
        const int64_t b = item.b0 + threadIdx.x;
        const double* ep = rebase(C.fa.e_part, a.ws) + b * tps;
        double e = 0.0;
        for (int64_t t = 0; t < tps; ++t) e += ep[t];
        const int64_t s = C.sample_off + b;
        a.E[s] = e;
        double g = 1.0, lt = e;
        if (C.loss_kind == 1) {
          const double dd = e - (double)a.y[s];
          g = 2.0 * dd * C.inv_B;
          lt = dd * dd * C.inv_B;
        }
        const_cast<double*>(rebase(C.ba.dLdE, a.ws))[b] = g;  // the item's own workspace row
        a.lterm[s] = lt;
      }
      __syncthreads();
    }
    for (int p = 0; p < C.n_bwd; ++p) {
      load_args(s_a, C.ba, C.bwd[p], a.ws);
      run_item_pass(true, s_a, item.b0);
    }
  }
}

// grad[o], o over every circuit's parameters: one warp per value, fixed order.
__global__ void batch_g_reduce_kernel(const BatchArgs a, int64_t n_out) {
  const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= n_out) return;
  const int c = find_circuit(a.grad_out_off, a.n_circ, o);
  const BatchCircuit& C = a.circ[c];
  const int p = (int)(o - a.grad_out_off[c]);
  const double* gp = rebase(C.ba.g_part, a.ws);
  const int64_t rows = C.ba.g_accum ? C.ba.B : (C.ba.B << C.ba.tps_log2);
  double s = 0.0;
  for (int k = C.param_off[p]; k < C.param_off[p + 1]; ++k) {
    const int term = C.param_terms[k];
    for (int64_t r = lane; r < rows; r += 32) s += gp[r * C.ba.n_slots + term];
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) a.grad[C.grad_off + p] = s;
}

__global__ void batch_loss_kernel(const BatchArgs a) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < a.n_samples; i += blockDim.x) s += a.lterm[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) a.loss[0] = red[0];
}

cudaError_t opt_in(const void* fn, size_t smem, OptIn& o) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tab = dev >= 0 && dev < 64;
  if (tab && o.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && tab) o.done[dev].store(true, std::memory_order_release);
  return e;
}

int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const bool tab = dev >= 0 && dev < 64;
  if (tab) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (tab) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int64_t stream_grid(int64_t want) {
  const int64_t cap = 16ll * device_sms();
  return cap > 0 && want > cap ? cap : want;
}

int batch_grid() { return 2 * device_sms(); }

cudaError_t launch_batch(const BatchArgs& a, int grid, int64_t prep_total, int64_t n_grad_out, cudaStream_t st) {
  static OptIn once;
  const size_t smem = 2 * (size_t)kTileAmps * sizeof(float2);
  cudaError_t e = opt_in(reinterpret_cast<const void*>(batch_kernel), smem, once);
  if (e != cudaSuccess) return e;
  if (prep_total > 0) batch_prep_kernel<<<(unsigned)((prep_total + 63) / 64), 64, 0, st>>>(a, prep_total);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.queue, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
  if (a.n_items > 0) {
    const int g = grid < a.n_items ? grid : a.n_items;
    batch_kernel<<<(unsigned)g, kThreads, smem, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (n_grad_out > 0) batch_g_reduce_kernel<<<(unsigned)((n_grad_out * 32 + 255) / 256), 256, 0, st>>>(a, n_grad_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  batch_loss_kernel<<<1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---- launchers ----------------------------------------------------------------
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t st) {
  int64_t total = (int64_t)a.n_fused + a.n_terms + (int64_t)a.B * a.n_eff + round_par_elems(a);
  if (total == 0 && !a.zero_word) return cudaSuccess;
  if (total == 0) total = 1;  // element 0 only clears the counter
  // float64 work per element: small blocks spread it over more SMs
  const int blk = 64;
  prep_kernel<<<(unsigned)((total + blk - 1) / blk), blk, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pass(bool bwd, const PassArgs& a, cudaStream_t st, int fwd_ctas) {
  const int tiles_per_cta = kThreads >> (a.pd.K - kRegBits);
  const int64_t total_tiles = (int64_t)a.B << a.tps_log2;
  const int64_t grid = (total_tiles + tiles_per_cta - 1) / tiles_per_cta;
  if (grid == 0) return cudaSuccess;
  const size_t smem = (size_t)(bwd ? 2 : 1) * kTileAmps * sizeof(float2);
  const bool rounds = a.rounds != nullptr, rx = rounds && a.rx_items;
  if (bwd) {
    // 64 KiB of dynamic shared memory needs the opt-in
    static OptIn once_generic, once_rounds, once_rx;
    cudaError_t e = rx       ? opt_in(reinterpret_cast<const void*>(pass_kernel<true, true, true>), smem, once_rx)
                    : rounds ? opt_in(reinterpret_cast<const void*>(pass_kernel<true, true>), smem, once_rounds)
                             : opt_in(reinterpret_cast<const void*>(pass_kernel<true, false>), smem, once_generic);
    if (e != cudaSuccess) return e;
    if (rx) pass_kernel<true, true, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
    else if (rounds) pass_kernel<true, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
    else pass_kernel<true, false><<<(unsigned)grid, kThreads, smem, st>>>(a);
  } else {
    // more tiles than two CTAs per SM hold: the three-CTA round instances
    // (fewer registers, more warps to hide latency across the waves)
    const int n_sm = device_sms();
    if (n_sm == 0) return cudaErrorInvalidDevice;
    const bool three = rounds && (fwd_ctas == 3 || (fwd_ctas == 0 && grid > 2ll * n_sm));
    if (rx && three) pass_kernel<false, true, true, 3><<<(unsigned)grid, kThreads, smem, st>>>(a);
    else if (rx) pass_kernel<false, true, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
    else if (three) pass_kernel<false, true, false, 3><<<(unsigned)grid, kThreads, smem, st>>>(a);
    else if (rounds) pass_kernel<false, true><<<(unsigned)grid, kThreads, smem, st>>>(a);
    else pass_kernel<false, false><<<(unsigned)grid, kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

// ---- observables whose X/Y qubits lie outside the tile (App. B.2) ---------------
// E partials: CTA (b, t) sums Re(conj(a_x) (O a)_x) over amplitudes
// x in [t*4096, (t+1)*4096) of sample b, with (O a)_x = i^{#Y} (-1)^{|(x^xm)&zm|} a_{x^xm};
// one fp64 partial per CTA, the same [B][rows] layout as the pass kernels.
__global__ void __launch_bounds__(kThreads) expect_full_kernel(const float2* psi, int n_eff, int64_t rows,
                                                               uint32_t xm, uint32_t zm, uint32_t yc,
                                                               double* e_part) {
  __shared__ double red[kThreads / 32];
  const int64_t dim = 1ll << n_eff;
  const int64_t chunk = dim / rows;
  const int64_t b = blockIdx.x / rows, t = blockIdx.x - b * rows;
  const float2* s = psi + b * dim;
  float acc = 0.f;
  for (int64_t k = threadIdx.x; k < chunk; k += kThreads) {
    const uint32_t x = (uint32_t)(t * chunk + k), xp = x ^ xm;
    const float2 v = s[x];
    const float2 w = mul_ipow(s[xp], yc);
    acc += flip(v.x * w.x + v.y * w.y, __popc(xp & zm) & 1u);
  }
  double d = (double)acc;
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) sum += red[w];
    e_part[blockIdx.x] = sum;
  }
}

// Adjoint seed lambda_x = 2 (dL/dE_b) (O psi_M)_x (Eq. 4) for every amplitude.
__global__ void seed_full_kernel(const float2* psi, float2* lam, int n_eff, int64_t B, uint32_t xm, uint32_t zm,
                                 uint32_t yc, const double* dLdE) {
  const int64_t dim = 1ll << n_eff;
  const int64_t total = B * dim;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i >> n_eff;
    const uint32_t x = (uint32_t)(i & (dim - 1)), xp = x ^ xm;
    const float scale = (float)(2.0 * dLdE[b]);
    const float2 v = mul_ipow(psi[b * dim + xp], yc);
    const uint32_t sg = __popc(xp & zm) & 1u;
    lam[i] = make_float2(flip(v.x, sg) * scale, flip(v.y, sg) * scale);
  }
}

cudaError_t launch_expect_full(const float2* psi, int n_eff, int64_t B, int64_t rows, uint32_t xm, uint32_t zm,
                               uint32_t yc, double* e_part, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  expect_full_kernel<<<(unsigned)(B * rows), kThreads, 0, st>>>(psi, n_eff, rows, xm, zm, yc, e_part);
  return cudaGetLastError();
}

cudaError_t launch_seed_full(const float2* psi, float2* lam, int n_eff, int64_t B, uint32_t xm, uint32_t zm,
                             uint32_t yc, const double* dLdE, cudaStream_t st) {
  const int64_t total = B << n_eff;
  if (total == 0) return cudaSuccess;
  const int64_t want = (total + kThreads - 1) / kThreads;
  const unsigned grid = (unsigned)stream_grid(want);
  seed_full_kernel<<<grid, kThreads, 0, st>>>(psi, lam, n_eff, B, xm, zm, yc, dLdE);
  return cudaGetLastError();
}

cudaError_t launch_pass_tc(const PassArgs& a, cudaStream_t st) {
  if (a.pd.K != kMaxTileBits || a.rounds == nullptr || a.tcb == nullptr) return cudaErrorInvalidValue;
  const int64_t grid = (int64_t)a.B << a.tps_log2;
  if (grid == 0) return cudaSuccess;
  const size_t smem = (size_t)kTileAmps * sizeof(float2) + (size_t)2 * kMaxStepRounds * kTcBFloats * sizeof(float);
  static OptIn once;
  cudaError_t e = opt_in(reinterpret_cast<const void*>(tc_pass_kernel), smem, once);
  if (e != cudaSuccess) return e;
  tc_pass_kernel<<<(unsigned)grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tc_tables(const uint4* fwd_rounds, int32_t n_rounds, const double* mats64, float* tcb,
                             cudaStream_t st) {
  const int64_t total = (int64_t)n_rounds * 1024;
  if (total == 0) return cudaSuccess;
  tc_table_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(fwd_rounds, n_rounds, mats64, tcb);
  return cudaGetLastError();
}

// Failure-path check of the bounded waits: one thread waits on an mbarrier
// that nothing arrives at, gives up after `limit` polls and records the
// timeout in the device error word, exactly as the tensor-core path would.
__global__ void bounded_wait_probe_kernel(long long limit) {
  __shared__ __align__(8) uint64_t mbar;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const uint32_t addr = smem_u32(&mbar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(0u)
        : "memory");
    if (done) return;
  }
  atomicExch(&g_qf_device_status, 1);
}

cudaError_t bounded_wait_probe(long long limit, cudaStream_t st) {
  if (limit < 1 || limit > (1ll << 20)) return cudaErrorInvalidValue;
  bounded_wait_probe_kernel<<<1, 1, 0, st>>>(limit);
  return cudaGetLastError();
}

cudaError_t device_status(int32_t* code, cudaStream_t st) {
  int32_t v = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_qf_device_status, sizeof(v), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *code = v;
  const int32_t zero = 0;
  e = cudaMemcpyToSymbolAsync(g_qf_device_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t launch_e_reduce(const double* e_part, int64_t B, int tps, double* E, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  if (tps >= 256) e_reduce_block_kernel<<<(unsigned)B, 256, 0, st>>>(e_part, tps, E);
  else e_reduce_kernel<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(e_part, B, tps, E);
  return cudaGetLastError();
}

cudaError_t launch_g_reduce(const GradReduceArgs& a, cudaStream_t st) {
  const int64_t n = a.per_sample ? (int64_t)a.B * a.n_params : a.n_params;
  if (n == 0) return cudaSuccess;
  GradReduceArgs r = a;
  if (g_reduce_stages(a.tps, a.slot_step) == 2) {
    // many rows per output: coalesced chunk sums first (groups: the samples
    // in per-sample mode, else all rows), then the fixed-order sum over chunks
    if (a.scratch == nullptr || a.B == 0) return cudaErrorInvalidValue;
    const int64_t groups = a.per_sample ? a.B : 1;
    const int64_t rows = a.per_sample ? a.tps : a.B * a.tps;
    const int64_t chunks = (rows + kGReduceChunk - 1) / kGReduceChunk;
    const int S = (int)a.slot_stride;
    const dim3 grid((unsigned)(groups * chunks), (unsigned)((S + 255) / 256));
    g_partial_kernel<<<grid, 256, 0, st>>>(a.g_part, rows, chunks, a.slot_stride, S, a.scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    r.g_part = a.scratch;
    r.B = groups;
    r.tps = chunks;
    r.per_sample = a.per_sample;
  }
  const int64_t threads = n * 32;
  g_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(r);
  return cudaGetLastError();
}

cudaError_t launch_loss(int kind, const double* E, const float* y, int64_t B, double* loss, double* dLdE,
                        cudaStream_t st) {
  loss_kernel<float><<<1, 256, 0, st>>>(kind, const_cast<double*>(E), y, B, B > 0 ? 2.0 / (double)B : 0.0, loss,
                                         dLdE, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_loss64(int kind, const double* E, const double* y, int64_t B, double* loss, double* dLdE,
                          cudaStream_t st) {
  loss_kernel<double><<<1, 256, 0, st>>>(kind, const_cast<double*>(E), y, B, B > 0 ? 2.0 / (double)B : 0.0, loss,
                                          dLdE, nullptr, 0);
  return cudaGetLastError();
}

bool e_loss_fusable(int64_t B, int tps) { return tps < 256 && B * tps <= 65536; }

template <class Y>
static cudaError_t launch_e_loss_t(const double* e_part, int tps, int kind, double* E, const Y* y, int64_t B,
                                   double* loss, double* dLdE, cudaStream_t st) {
  loss_kernel<Y><<<1, 256, 0, st>>>(kind, E, y, B, B > 0 ? 2.0 / (double)B : 0.0, loss, dLdE, e_part, tps);
  return cudaGetLastError();
}

cudaError_t launch_e_loss(const double* e_part, int tps, int kind, double* E, const float* y, int64_t B,
                          double* loss, double* dLdE, cudaStream_t st) {
  return launch_e_loss_t<float>(e_part, tps, kind, E, y, B, loss, dLdE, st);
}

cudaError_t launch_e_loss64(const double* e_part, int tps, int kind, double* E, const double* y, int64_t B,
                            double* loss, double* dLdE, cudaStream_t st) {
  return launch_e_loss_t<double>(e_part, tps, kind, E, y, B, loss, dLdE, st);
}

}  // namespace qf
