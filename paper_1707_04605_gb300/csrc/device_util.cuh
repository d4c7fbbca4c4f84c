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
__device__ __forceinline__ float4 leap(float4 c, float4 self, float4 old, float4 acc) {
  float4 o;
  o.x = c.x * self.x - c.y * old.x - c.z * acc.x;
  o.y = c.x * self.y - c.y * old.y - c.z * acc.y;
  o.z = c.x * self.z - c.y * old.z - c.z * acc.z;
  o.w = c.x * self.w - c.y * old.w - c.z * acc.w;
  return o;
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
