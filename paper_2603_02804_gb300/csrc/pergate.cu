// Unfused comparator: one kernel launch per gate, forward and backward.
//
// This is the memory-efficient per-gate adjoint the paper cites as prior art
// (Sec. 1: un-apply each gate sequentially in the backward, one full pass over
// the state per gate). Every kernel is coalesced and vectorised (float4 = two
// amplitudes) so the fused path is compared with a well-written baseline, not
// a strawman. Checkpointed states re-anchor psi exactly as in the fused path.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace qf {

namespace {

constexpr int kPgThreads = 256;

__device__ __forceinline__ float flip(float v, uint32_t s) {
  return __int_as_float(__float_as_int(v) ^ (int)(s << 31));
}

// index with a zero inserted at bit position q
__device__ __forceinline__ uint64_t ins0(uint64_t i, int q) {
  const uint64_t lo = i & ((1ull << q) - 1);
  return ((i >> q) << (q + 1)) | lo;
}

__device__ __forceinline__ float2 mul_ipow(float2 v, uint32_t k) {
  switch (k & 3u) {
    case 0: return v;
    case 1: return make_float2(-v.y, v.x);
    case 2: return make_float2(-v.x, -v.y);
    default: return make_float2(v.y, -v.x);
  }
}

// 2x2 rotation u(t) = c I - i s P applied to (a0, a1); adj = u^dagger.
template <int KIND, bool ADJ>
__device__ __forceinline__ void rot(float2& a0, float2& a1, float c, float s) {
  const float ss = ADJ ? -s : s;  // u^dagger = u(-t)
  if (KIND == G_RZ) {
    a0 = make_float2(c * a0.x + ss * a0.y, c * a0.y - ss * a0.x);
    a1 = make_float2(c * a1.x - ss * a1.y, c * a1.y + ss * a1.x);
  } else if (KIND == G_RY) {
    const float2 x = a0, y = a1;
    a0 = make_float2(c * x.x - ss * y.x, c * x.y - ss * y.y);
    a1 = make_float2(ss * x.x + c * y.x, ss * x.y + c * y.y);
  } else {
    const float2 x = a0, y = a1;
    a0 = make_float2(c * x.x + ss * y.y, c * x.y - ss * y.x);
    a1 = make_float2(c * y.x + ss * x.y, c * y.y - ss * x.x);
  }
}

// Im <l|P|p> over one pair
template <int KIND>
__device__ __forceinline__ float imp(float2 p0, float2 p1, float2 l0, float2 l1) {
  if (KIND == G_RZ) return l0.x * p0.y - l0.y * p0.x - l1.x * p1.y + l1.y * p1.x;
  if (KIND == G_RY) return l1.x * p0.x + l1.y * p0.y - l0.x * p1.x - l0.y * p1.y;
  return l0.x * p1.y - l0.y * p1.x + l1.x * p0.y - l1.y * p0.x;
}

__global__ void pg_encode_kernel(const PerGateArgs a, const float2* enc) {
  const int64_t dim = 1ll << a.n_eff;
  const int64_t npair = (int64_t)a.B * (dim >> 1);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npair;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = p / (dim >> 1);
    const uint64_t x = (uint64_t)(p - b * (dim >> 1)) * 2;
    const float2* e = enc + b * a.n_eff;
    float pr = 1.f;
    for (int q = 1; q < a.n_eff; ++q) pr *= ((x >> q) & 1) ? e[q].y : e[q].x;
    reinterpret_cast<float4*>(a.psi + b * dim)[x >> 1] = make_float4(pr * e[0].x, 0.f, pr * e[0].y, 0.f);
  }
}

// Given initial states [B][2^n_in] into [B][2^n_eff] (padding qubits |0>).
__global__ void pg_load_states_kernel(const PerGateArgs a, const float2* in, int n_in) {
  const int64_t dim = 1ll << a.n_eff, din = 1ll << n_in;
  const int64_t total = (int64_t)a.B * dim;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / dim, x = i - b * dim;
    a.psi[i] = x < din ? in[b * din + x] : make_float2(0.f, 0.f);
  }
}

// CNOT(c, t): swap the amplitude pairs over bit t whose bit c is 1 (psi, and
// lambda when both): self-inverse, no gradient.
__global__ void pg_cnot_kernel(const PerGateArgs a, int c, int t, int both) {
  const int64_t dim = 1ll << a.n_eff;
  const int64_t per = dim >> 2;  // pairs with bit c = 1
  const int64_t total = (int64_t)a.B * per;
  const int lo = c < t ? c : t, hi = c < t ? t : c;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / per;
    uint64_t k = (uint64_t)(i - b * per);
    // insert zero bits at lo and hi, then set the control bit
    k = ((k >> lo) << (lo + 1)) | (k & ((1ull << lo) - 1));
    k = ((k >> hi) << (hi + 1)) | (k & ((1ull << hi) - 1));
    const uint64_t x0 = k | (1ull << c), x1 = x0 | (1ull << t);
    float2* p = a.psi + b * dim;
    const float2 u = p[x0];
    p[x0] = p[x1];
    p[x1] = u;
    if (both) {
      float2* q = a.lam + b * dim;
      const float2 v = q[x0];
      q[x0] = q[x1];
      q[x1] = v;
    }
  }
}

template <int KIND>
__global__ void pg_rot_kernel(const PerGateArgs a, int q, const float2* cs, int slot) {
  const float2 csv = __ldg(cs + slot);
  const int64_t dim = 1ll << a.n_eff;
  if (q == 0) {
    const int64_t n = (int64_t)a.B * (dim >> 1);
    float4* v = reinterpret_cast<float4*>(a.psi);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
      float4 w = v[p];
      float2 a0 = make_float2(w.x, w.y), a1 = make_float2(w.z, w.w);
      rot<KIND, false>(a0, a1, csv.x, csv.y);
      v[p] = make_float4(a0.x, a0.y, a1.x, a1.y);
    }
  } else {
    // each thread: the float4 at x (bit q = 0) and its partner x | 2^q
    const int64_t n = (int64_t)a.B * (dim >> 2);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
      const int64_t b = p / (dim >> 2);
      const uint64_t x = ins0((uint64_t)(p - b * (dim >> 2)) * 2, q);
      float4* v0 = reinterpret_cast<float4*>(a.psi + b * dim + x);
      float4* v1 = reinterpret_cast<float4*>(a.psi + b * dim + (x | (1ull << q)));
      float4 w0 = *v0, w1 = *v1;
      float2 a0 = make_float2(w0.x, w0.y), a1 = make_float2(w1.x, w1.y);
      float2 c0 = make_float2(w0.z, w0.w), c1 = make_float2(w1.z, w1.w);
      rot<KIND, false>(a0, a1, csv.x, csv.y);
      rot<KIND, false>(c0, c1, csv.x, csv.y);
      *v0 = make_float4(a0.x, a0.y, c0.x, c0.y);
      *v1 = make_float4(a1.x, a1.y, c1.x, c1.y);
    }
  }
}

// CZ on the quarter of the amplitudes it touches (bits c and t both set).
__global__ void pg_cz_kernel(const PerGateArgs a, int c, int t, int both) {
  const int64_t dim = 1ll << a.n_eff;
  const int lo = c < t ? c : t, hi = c < t ? t : c;
  const int64_t per = dim >> 2;
  const int64_t n = (int64_t)a.B * per;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = p / per;
    const uint64_t x = ins0(ins0((uint64_t)(p - b * per), lo), hi) | (1ull << lo) | (1ull << hi);
    float2* s = a.psi + b * dim + x;
    *s = make_float2(-s->x, -s->y);
    if (both) {
      float2* l = a.lam + b * dim + x;
      *l = make_float2(-l->x, -l->y);
    }
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kPgThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kPgThreads / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// grid (chunks, B): E partial of chunk of sample b
__global__ void pg_expect_kernel(const PerGateArgs a, uint32_t xm, uint32_t zm, uint32_t yc, double* e_part) {
  const int64_t dim = 1ll << a.n_eff;
  const int64_t b = blockIdx.y;
  const int64_t per = dim / a.chunks;
  const float2* s = a.psi + b * dim;
  float acc = 0.f;
  for (int64_t x = blockIdx.x * per + threadIdx.x; x < (int64_t)(blockIdx.x + 1) * per; x += blockDim.x) {
    const uint64_t xp = (uint64_t)x ^ xm;
    const float2 v = s[x];
    const float2 w = mul_ipow(s[xp], yc);
    acc += flip(v.x * w.x + v.y * w.y, __popcll(xp & zm) & 1u);
  }
  const double t = block_sum((double)acc);
  if (threadIdx.x == 0) e_part[b * a.chunks + blockIdx.x] = t;
}

__global__ void pg_seed_kernel(const PerGateArgs a, uint32_t xm, uint32_t zm, uint32_t yc, const double* dLdE) {
  const int64_t dim = 1ll << a.n_eff;
  const int64_t n = (int64_t)a.B * dim;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / dim;
    const uint64_t x = (uint64_t)(i - b * dim), xp = x ^ xm;
    const float sc = (float)(2.0 * dLdE[b]);
    const float2 w = mul_ipow(a.psi[b * dim + xp], yc);
    const uint32_t sg = __popcll(xp & zm) & 1u;
    a.lam[i] = make_float2(flip(w.x, sg) * sc, flip(w.y, sg) * sc);
  }
}

// grid (chunks, B). Per pair: grad partial from (psi_j, lambda_j), then
// psi <- u^dagger psi, lambda <- u^dagger lambda.
template <int KIND>
__global__ void pg_rot_bwd_kernel(const PerGateArgs a, int q, const float2* cs, int slot, double* g_part) {
  const float2 csv = __ldg(cs + slot);
  const int64_t dim = 1ll << a.n_eff;
  const int64_t b = blockIdx.y;
  float2* ps = a.psi + b * dim;
  float2* ls = a.lam + b * dim;
  float acc = 0.f;
  if (q == 0) {
    const int64_t per = (dim >> 1) / a.chunks;
    for (int64_t p = blockIdx.x * per + threadIdx.x; p < (int64_t)(blockIdx.x + 1) * per; p += blockDim.x) {
      float4 w = reinterpret_cast<float4*>(ps)[p], m = reinterpret_cast<float4*>(ls)[p];
      float2 p0 = make_float2(w.x, w.y), p1 = make_float2(w.z, w.w);
      float2 l0 = make_float2(m.x, m.y), l1 = make_float2(m.z, m.w);
      acc += imp<KIND>(p0, p1, l0, l1);
      rot<KIND, true>(p0, p1, csv.x, csv.y);
      rot<KIND, true>(l0, l1, csv.x, csv.y);
      reinterpret_cast<float4*>(ps)[p] = make_float4(p0.x, p0.y, p1.x, p1.y);
      reinterpret_cast<float4*>(ls)[p] = make_float4(l0.x, l0.y, l1.x, l1.y);
    }
  } else {
    const int64_t per = (dim >> 2) / a.chunks;
    for (int64_t p = blockIdx.x * per + threadIdx.x; p < (int64_t)(blockIdx.x + 1) * per; p += blockDim.x) {
      const uint64_t x = ins0((uint64_t)p * 2, q), y = x | (1ull << q);
      float4 w0 = *reinterpret_cast<float4*>(ps + x), w1 = *reinterpret_cast<float4*>(ps + y);
      float4 m0 = *reinterpret_cast<float4*>(ls + x), m1 = *reinterpret_cast<float4*>(ls + y);
      float2 p0 = make_float2(w0.x, w0.y), p1 = make_float2(w1.x, w1.y);
      float2 r0 = make_float2(w0.z, w0.w), r1 = make_float2(w1.z, w1.w);
      float2 l0 = make_float2(m0.x, m0.y), l1 = make_float2(m1.x, m1.y);
      float2 k0 = make_float2(m0.z, m0.w), k1 = make_float2(m1.z, m1.w);
      acc += imp<KIND>(p0, p1, l0, l1) + imp<KIND>(r0, r1, k0, k1);
      rot<KIND, true>(p0, p1, csv.x, csv.y);
      rot<KIND, true>(r0, r1, csv.x, csv.y);
      rot<KIND, true>(l0, l1, csv.x, csv.y);
      rot<KIND, true>(k0, k1, csv.x, csv.y);
      *reinterpret_cast<float4*>(ps + x) = make_float4(p0.x, p0.y, r0.x, r0.y);
      *reinterpret_cast<float4*>(ps + y) = make_float4(p1.x, p1.y, r1.x, r1.y);
      *reinterpret_cast<float4*>(ls + x) = make_float4(l0.x, l0.y, k0.x, k0.y);
      *reinterpret_cast<float4*>(ls + y) = make_float4(l1.x, l1.y, k1.x, k1.y);
    }
  }
  const double t = block_sum((double)acc);
  if (threadIdx.x == 0) g_part[b * a.chunks + blockIdx.x] = 0.5 * t;
}

__global__ void pg_copy_kernel(const float4* src, float4* dst, int64_t n4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

unsigned grid_for(int64_t n) {
  const int64_t g = stream_grid((n + kPgThreads - 1) / kPgThreads);
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// Partial rows per sample: one CTA per 8192 amplitudes (at least one).
int32_t pg_chunks(int32_t n_eff) {
  const int e = n_eff - 13;
  return e > 0 ? (1 << e) : 1;
}

cudaError_t pg_encode(const PerGateArgs& a, const float2* enc, cudaStream_t st) {
  pg_encode_kernel<<<grid_for(a.B << (a.n_eff - 1)), kPgThreads, 0, st>>>(a, enc);
  return cudaGetLastError();
}

cudaError_t pg_load_states(const PerGateArgs& a, const float2* in, int n_in, cudaStream_t st) {
  pg_load_states_kernel<<<grid_for(a.B << a.n_eff), kPgThreads, 0, st>>>(a, in, n_in);
  return cudaGetLastError();
}

cudaError_t pg_rot(const PerGateArgs& a, int kind, int q, const float2* cs, int slot, cudaStream_t st) {
  const int64_t dim = 1ll << a.n_eff;
  const unsigned g = grid_for(q == 0 ? a.B * (dim >> 1) : a.B * (dim >> 2));
  if (kind == G_RZ) pg_rot_kernel<G_RZ><<<g, kPgThreads, 0, st>>>(a, q, cs, slot);
  else if (kind == G_RY) pg_rot_kernel<G_RY><<<g, kPgThreads, 0, st>>>(a, q, cs, slot);
  else pg_rot_kernel<G_RX><<<g, kPgThreads, 0, st>>>(a, q, cs, slot);
  return cudaGetLastError();
}

cudaError_t pg_cnot(const PerGateArgs& a, int c, int t, bool both, cudaStream_t st) {
  pg_cnot_kernel<<<grid_for(a.B << (a.n_eff - 2)), kPgThreads, 0, st>>>(a, c, t, both ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t pg_cz(const PerGateArgs& a, int c, int t, bool both, cudaStream_t st) {
  pg_cz_kernel<<<grid_for(a.B << (a.n_eff - 2)), kPgThreads, 0, st>>>(a, c, t, both ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t pg_expect(const PerGateArgs& a, uint32_t x_mask, uint32_t z_mask, uint32_t y_count,
                      double* e_part, cudaStream_t st) {
  if (a.B == 0) return cudaSuccess;
  pg_expect_kernel<<<dim3((unsigned)a.chunks, (unsigned)a.B), kPgThreads, 0, st>>>(a, x_mask, z_mask, y_count,
                                                                                   e_part);
  return cudaGetLastError();
}

cudaError_t pg_seed(const PerGateArgs& a, uint32_t x_mask, uint32_t z_mask, uint32_t y_count,
                    const double* dLdE, cudaStream_t st) {
  pg_seed_kernel<<<grid_for(a.B << a.n_eff), kPgThreads, 0, st>>>(a, x_mask, z_mask, y_count, dLdE);
  return cudaGetLastError();
}

cudaError_t pg_rot_bwd(const PerGateArgs& a, int kind, int q, const float2* cs, int slot, double* g_part,
                       cudaStream_t st) {
  if (a.B == 0) return cudaSuccess;
  const dim3 g((unsigned)a.chunks, (unsigned)a.B);
  if (kind == G_RZ) pg_rot_bwd_kernel<G_RZ><<<g, kPgThreads, 0, st>>>(a, q, cs, slot, g_part);
  else if (kind == G_RY) pg_rot_bwd_kernel<G_RY><<<g, kPgThreads, 0, st>>>(a, q, cs, slot, g_part);
  else pg_rot_bwd_kernel<G_RX><<<g, kPgThreads, 0, st>>>(a, q, cs, slot, g_part);
  return cudaGetLastError();
}

cudaError_t pg_copy(const float2* src, float2* dst, int64_t n, cudaStream_t st) {
  const int64_t n4 = n / 2;
  pg_copy_kernel<<<grid_for(n4), kPgThreads, 0, st>>>(reinterpret_cast<const float4*>(src),
                                                     reinterpret_cast<float4*>(dst), n4);
  return cudaGetLastError();
}

}  // namespace qf
