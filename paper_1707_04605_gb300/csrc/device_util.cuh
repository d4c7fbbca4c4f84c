// Small device helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "mg_internal.h"

namespace mg {
namespace dev {

constexpr int kWarps = 8;            // warps per block of the batched kernels
constexpr int kThreads = 32 * kWarps;
constexpr int kTile = 128;           // shots per source tile

__device__ __forceinline__ float4 ld4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4v(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st4(float* p, float4 v) {
  *reinterpret_cast<float4*>(p) = v;
}
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z),
                     fmaf(a, x.w, y.w));
}
// Component d (0..3) of a float4 without dynamic register indexing.
__device__ __forceinline__ void add_comp(float4& v, int d, float x) {
  v.x += d == 0 ? x : 0.0f;
  v.y += d == 1 ? x : 0.0f;
  v.z += d == 2 ? x : 0.0f;
  v.w += d == 3 ? x : 0.0f;
}
__device__ __forceinline__ float get_comp(const float4& v, int d) {
  return d == 0 ? v.x : d == 1 ? v.y : d == 2 ? v.z : v.w;
}

__device__ __forceinline__ float4 scale4(float a, float4 x) {
  return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
}

// out = alpha self - beta old - gamma acc
// The per-row combinations below are written with explicit round-to-nearest
// intrinsics so that every kernel variant (row, tiled, multi-instance; any
// launch shape) performs the same floating-point operations in the same
// order, leaving the compiler no freedom to contract them differently.

// out = alpha self - beta old - gamma acc, evaluated as
// fma(-gamma, acc, fma(alpha, self, -(beta old))).
__device__ __forceinline__ float leap1(float a, float b, float g, float self, float old,
                                       float acc) {
  return __fmaf_rn(-g, acc, __fmaf_rn(a, self, -__fmul_rn(b, old)));
}
__device__ __forceinline__ float4 leap(float4 c, float4 self, float4 old, float4 acc) {
  return make_float4(leap1(c.x, c.y, c.z, self.x, old.x, acc.x),
                     leap1(c.x, c.y, c.z, self.y, old.y, acc.y),
                     leap1(c.x, c.y, c.z, self.z, old.z, acc.z),
                     leap1(c.x, c.y, c.z, self.w, old.w, acc.w));
}

// Second and centred time differences of a state at one node.
__device__ __forceinline__ float d2t(float next, float cur, float prev) {
  return __fadd_rn(__fmaf_rn(-2.0f, cur, next), prev);
}
__device__ __forceinline__ float d1t(float next, float prev) { return __fsub_rn(next, prev); }

// Tangent correction: dq+ -= cm (p+ - 2p + p-) + cd (p+ - p-).
__device__ __forceinline__ float4 tangent_fix(float4 qn, float4 pn, float4 ps, float4 pold,
                                              float2 tc) {
#define MG_TF(X) \
  qn.X = __fsub_rn(qn.X, __fmaf_rn(tc.x, d2t(pn.X, ps.X, pold.X), __fmul_rn(tc.y, d1t(pn.X, pold.X))));
  MG_TF(x) MG_TF(y) MG_TF(z) MG_TF(w)
#undef MG_TF
  return qn;
}

// Adjoint time-sum terms of one float4 of shots:
// t1 += p_k (mu_{k-1} - 2 mu_k + mu_{k+1}),  t2 += p_k (mu_{k-1} - mu_{k+1}).
__device__ __forceinline__ void adj_terms(float4 pk, float4 out, float4 self, float4 old,
                                          float& t1, float& t2) {
#define MG_AT(X) \
  t1 = __fmaf_rn(pk.X, d2t(out.X, self.X, old.X), t1); \
  t2 = __fmaf_rn(pk.X, d1t(out.X, old.X), t2);
  MG_AT(x) MG_AT(y) MG_AT(z) MG_AT(w)
#undef MG_AT
}

__device__ __forceinline__ void kahan_add(float* s, float* c, float term) {
  const float y = term - *c;
  const float t = *s + y;
  *c = (t - *s) - y;
  *s = t;
}

inline int check_launch() {
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

}  // namespace dev
}  // namespace mg
