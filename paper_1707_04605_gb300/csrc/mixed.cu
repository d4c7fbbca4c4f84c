// The paper's first-order leapfrog with element flux variables and the
// split-field perfectly matched layer (App. A, Eqs. (system1), (system2),
// (leap-frog1), (leap-frog2)).
//
//   q^(k)_{l+1/2} = (1 - dt zeta^(k)) q^(k)_{l-1/2} + dt sum_a dphi_a/dx_k p_l[a]   (per cell)
//   p_{l+1}       = p_l + dt/C (f_l - (R + S) p_l - sum_k B^(k)T q^(k)_{l+1/2})      (per node)
//
// A_ii = |T_i|, B^(k)_{ij} = |T_i| dphi_j/dx_k, C the lumped eps-mass, R the
// lumped sigma-mass (the handle's conductivity), S the lumped xi-mass, and
// f_l = dt sum_{m <= l} s_m (the source is the time integral of the
// wavelet).  Natural outer boundary: the layer absorbs.  State: p [n][ld],
// q [d][m][ld] FP32 (ld = padded shot count); a thread advances one float4
// of shots of one node or one cell.  Sample l of a trace is p_{l+1}.
//
// Jacobians with respect to the cell permittivity (only C depends on it):
//  * tangent, in lockstep with the forward: the fluxes of dp follow the
//    same update; dp_{l+1} = dp_l + dt/C (-(R+S) dp_l - sum_k B^(k)T dq^(k))
//    - (dC/C)(p_{l+1} - p_l), dC the lumped mass of the direction;
//  * adjoint, backwards over checkpointed segments (p and q stored every
//    ckpt_every steps, each segment's p states recomputed into a buffer):
//    with a the adjoint of p_{l+1} (traces' weights at the receivers plus
//    what step l+1 sends back) and r = a dt / C, the scaled flux adjoint
//    Qt^(k) = Q^(k)/|e| becomes (1 - dt zeta_k) Qt^(k) - sum_a dphi_a/dx_k r[v_a],
//    p_l receives a - (R+S) r + dt sum_k B^(k)T Qt^(k), and the C-sensitivity
//    gathers -sum_l a (p_{l+1} - p_l) / C; the cell gradient is
//    |e|/(d+1) times its sum over the cell's vertices, restricted to a level.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/mgwave.h"
#include "kernels.cuh"
#include "mesh_view.h"
#include "mg_internal.h"

namespace mg {
namespace {

constexpr int kMaxDim = 3;

// Step kernels run as programmatic dependents of the previous kernel on
// the stream: each waits for it to complete (and its stores to be visible)
// before touching any state, then lets the next launch be scheduled.
__device__ __forceinline__ void pdl_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Step index of a launch: l, plus the device int *base when the launch is
// a node of a CUDA graph replayed once per chunk of steps (the graph moves
// the base at its end).  Read after pdl_sync.
struct StepRef {
  int l;
  const int* base;
};
__device__ __forceinline__ int step_of(const StepRef& s) { return s.base ? s.l + *s.base : s.l; }

// p states kept in slots of one buffer: p_l in slot l mod K (stride ns4
// float4), so that a launch finds its states from its step index alone;
// seg == nullptr: the launch's own state pointers.
struct Slots {
  float4* seg;
  int64_t ns4;
  int K;
};
__device__ __forceinline__ float4* slot_of(const Slots& s, int l) {
  return s.seg + (int64_t)(l % s.K) * s.ns4;
}

// per node: {dt / C_i, R_i + S_i}
__global__ void k_flux_coefs(CoefArgs c, const double* __restrict__ xi, double dt,
                             float2* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= c.n) return;
  double C = 0.0, RS = 0.0;
  for (int64_t q = c.nc_ptr[r]; q < c.nc_ptr[r + 1]; ++q) {
    const int e = c.nc_cell[q];
    C += c.eps[e] * c.nc_w[q];
    if (c.sigma) RS += c.sigma[e] * c.nc_w[q];
    if (xi) RS += xi[e] * c.nc_w[q];
  }
  out[r] = make_float2((float)(dt / C), (float)RS);
}

// q^(k) <- (1 - dt zeta_k) q^(k) + dt sum_a grad[a][k] p[v_a]
template <int D>
__global__ void k_flux_q(int64_t m, int ld4, const int32_t* __restrict__ cells,
                         const float* __restrict__ grad, const float* __restrict__ damp,
                         const float4* __restrict__ p, float4* __restrict__ q, float dt,
                         StepRef sr, Slots sl) {
  pdl_sync();
  if (sl.seg) p = slot_of(sl, step_of(sr));
  const int64_t total = m * ld4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / ld4;
    const int c4 = (int)(t - e * ld4);
    float4 pv[D + 1];
#pragma unroll
    for (int a = 0; a <= D; ++a) pv[a] = __ldg(p + (int64_t)__ldg(cells + e * (D + 1) + a) * ld4 + c4);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int a = 0; a <= D; ++a) {
        const float g = __ldg(grad + (e * (D + 1) + a) * D + k);
        acc.x = fmaf(g, pv[a].x, acc.x);
        acc.y = fmaf(g, pv[a].y, acc.y);
        acc.z = fmaf(g, pv[a].z, acc.z);
        acc.w = fmaf(g, pv[a].w, acc.w);
      }
      const float keep = 1.0f - dt * __ldg(damp + e * D + k);
      float4* qp = q + ((int64_t)k * m + e) * ld4 + c4;
      const float4 o = *qp;
      *qp = make_float4(fmaf(keep, o.x, dt * acc.x), fmaf(keep, o.y, dt * acc.y),
                        fmaf(keep, o.z, dt * acc.z), fmaf(keep, o.w, dt * acc.w));
    }
  }
}

// pout <- p + dt/C (f delta_src - (R+S) p - sum_{e ni i} sum_k w[e,i,k] q^(k)_e)
// (pout may be p); sources and traces of the row's shots
template <int D>
__global__ void k_flux_p(int64_t n, int64_t m, int ld4, const int64_t* __restrict__ nc_ptr,
                         const int32_t* __restrict__ nc_cell, const float* __restrict__ w,
                         const float2* __restrict__ coef, const float4* __restrict__ q,
                         const float4* p, float4* pout, const int32_t* __restrict__ src_ptr,
                         const int32_t* __restrict__ src_shot, const int32_t* __restrict__ rec_ptr,
                         const int32_t* __restrict__ rec_shot,
                         const int32_t* __restrict__ rec_trace, const float* __restrict__ fl,
                         float* __restrict__ traces, int nt, StepRef sr, Slots sl) {
  pdl_sync();
  const int l = step_of(sr);
  const float f = __ldg(fl + l);
  if (sl.seg) {   // p_l in slot l, p_{l+1} into the next slot
    pout = slot_of(sl, l);
    p = pout;
    pout += sl.ns4;
  }
  const int64_t total = n * ld4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld4;
    const int c4 = (int)(t - i * ld4);
    float4 bt = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t s = __ldg(nc_ptr + i); s < __ldg(nc_ptr + i + 1); ++s) {
      const int64_t e = __ldg(nc_cell + s);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float wk = __ldg(w + s * D + k);
        const float4 qv = __ldg(q + ((int64_t)k * m + e) * ld4 + c4);
        bt.x = fmaf(wk, qv.x, bt.x);
        bt.y = fmaf(wk, qv.y, bt.y);
        bt.z = fmaf(wk, qv.z, bt.z);
        bt.w = fmaf(wk, qv.w, bt.w);
      }
    }
    const float2 c = __ldg(coef + i);
    float4 rhs = make_float4(-bt.x, -bt.y, -bt.z, -bt.w);
    const int s0 = __ldg(src_ptr + i), s1 = __ldg(src_ptr + i + 1);
    for (int s = s0; s < s1; ++s) {
      const int d = __ldg(src_shot + s) - 4 * c4;
      if (d == 0) rhs.x += f;
      if (d == 1) rhs.y += f;
      if (d == 2) rhs.z += f;
      if (d == 3) rhs.w += f;
    }
    float4 pv = p[t];
    pv.x = fmaf(c.x, fmaf(-c.y, pv.x, rhs.x), pv.x);
    pv.y = fmaf(c.x, fmaf(-c.y, pv.y, rhs.y), pv.y);
    pv.z = fmaf(c.x, fmaf(-c.y, pv.z, rhs.z), pv.z);
    pv.w = fmaf(c.x, fmaf(-c.y, pv.w, rhs.w), pv.w);
    pout[t] = pv;
    const int r0 = __ldg(rec_ptr + i), r1 = __ldg(rec_ptr + i + 1);
    for (int r = r0; r < r1; ++r) {
      const int d = __ldg(rec_shot + r) - 4 * c4;
      if (d < 0 || d > 3) continue;
      const float v = d == 0 ? pv.x : d == 1 ? pv.y : d == 2 ? pv.z : pv.w;
      traces[(int64_t)__ldg(rec_trace + r) * nt + l] = v;
    }
  }
}

// C_i = sum_{e ni i} x[e] |e| / (d+1) in FP64 (x = eps, or a direction)
__global__ void k_flux_mass(CoefArgs c, const double* __restrict__ x, double* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= c.n) return;
  double s = 0.0;
  for (int64_t q = c.nc_ptr[r]; q < c.nc_ptr[r + 1]; ++q) s += x[c.nc_cell[q]] * c.nc_w[q];
  out[r] = s;
}

__global__ void k_flux_ratio(int64_t n, const double* __restrict__ dC, const double* __restrict__ C,
                             float* __restrict__ ratio) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) ratio[r] = (float)(dC[r] / C[r]);
}

// Tangent node update: p as in k_flux_p, and
// dp <- dp + dt/C (-(R+S) dp - sum B^T dq) - ratio (p_new - p_old); traces of dp.
template <int D>
__global__ void k_flux_p_tan(int64_t n, int64_t m, int ld4, const int64_t* __restrict__ nc_ptr,
                             const int32_t* __restrict__ nc_cell, const float* __restrict__ w,
                             const float2* __restrict__ coef, const float* __restrict__ ratio,
                             const float4* __restrict__ q, const float4* __restrict__ dq,
                             float4* __restrict__ p, float4* __restrict__ dp,
                             const int32_t* __restrict__ src_ptr,
                             const int32_t* __restrict__ src_shot,
                             const int32_t* __restrict__ rec_ptr,
                             const int32_t* __restrict__ rec_shot,
                             const int32_t* __restrict__ rec_trace,
                             const float* __restrict__ fl, float* __restrict__ traces, int nt,
                             StepRef sr) {
  pdl_sync();
  const int l = step_of(sr);
  const float f = __ldg(fl + l);
  const int64_t total = n * ld4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld4;
    const int c4 = (int)(t - i * ld4);
    float4 bt = make_float4(0.f, 0.f, 0.f, 0.f), dbt = bt;
    for (int64_t s = __ldg(nc_ptr + i); s < __ldg(nc_ptr + i + 1); ++s) {
      const int64_t e = __ldg(nc_cell + s);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float wk = __ldg(w + s * D + k);
        const int64_t at = ((int64_t)k * m + e) * ld4 + c4;
        const float4 qv = __ldg(q + at), dv = __ldg(dq + at);
        bt.x = fmaf(wk, qv.x, bt.x);
        bt.y = fmaf(wk, qv.y, bt.y);
        bt.z = fmaf(wk, qv.z, bt.z);
        bt.w = fmaf(wk, qv.w, bt.w);
        dbt.x = fmaf(wk, dv.x, dbt.x);
        dbt.y = fmaf(wk, dv.y, dbt.y);
        dbt.z = fmaf(wk, dv.z, dbt.z);
        dbt.w = fmaf(wk, dv.w, dbt.w);
      }
    }
    const float2 c = __ldg(coef + i);
    const float rt = __ldg(ratio + i);
    float4 rhs = make_float4(-bt.x, -bt.y, -bt.z, -bt.w);
    const int s0 = __ldg(src_ptr + i), s1 = __ldg(src_ptr + i + 1);
    for (int s = s0; s < s1; ++s) {
      const int d = __ldg(src_shot + s) - 4 * c4;
      if (d == 0) rhs.x += f;
      if (d == 1) rhs.y += f;
      if (d == 2) rhs.z += f;
      if (d == 3) rhs.w += f;
    }
    float4 pv = p[t], dv = dp[t];
    const float4 inc = make_float4(fmaf(-c.y, pv.x, rhs.x), fmaf(-c.y, pv.y, rhs.y),
                                   fmaf(-c.y, pv.z, rhs.z), fmaf(-c.y, pv.w, rhs.w));
    dv.x = fmaf(-rt, c.x * inc.x, fmaf(c.x, fmaf(-c.y, dv.x, -dbt.x), dv.x));
    dv.y = fmaf(-rt, c.x * inc.y, fmaf(c.x, fmaf(-c.y, dv.y, -dbt.y), dv.y));
    dv.z = fmaf(-rt, c.x * inc.z, fmaf(c.x, fmaf(-c.y, dv.z, -dbt.z), dv.z));
    dv.w = fmaf(-rt, c.x * inc.w, fmaf(c.x, fmaf(-c.y, dv.w, -dbt.w), dv.w));
    pv.x = fmaf(c.x, inc.x, pv.x);
    pv.y = fmaf(c.x, inc.y, pv.y);
    pv.z = fmaf(c.x, inc.z, pv.z);
    pv.w = fmaf(c.x, inc.w, pv.w);
    p[t] = pv;
    dp[t] = dv;
    const int r0 = __ldg(rec_ptr + i), r1 = __ldg(rec_ptr + i + 1);
    for (int r = r0; r < r1; ++r) {
      const int d = __ldg(rec_shot + r) - 4 * c4;
      if (d < 0 || d > 3) continue;
      const float v = d == 0 ? dv.x : d == 1 ? dv.y : d == 2 ? dv.z : dv.w;
      traces[(int64_t)__ldg(rec_trace + r) * nt + l] = v;
    }
  }
}

// Adjoint node kernel of reverse step l (p_l in slot l mod K of sl, p_{l+1}
// in the next slot).  a = adjoint of p_{l+1}: what step
// l+1 sent back (tp + dt sum_k B^(k)T Qt^(k); zero when l = nt-1) plus the
// weights of the row's receivers at sample l.  Sums a (p_{l+1} - p_l) over
// the node's shots in FP32 (the threads of a node are consecutive lanes:
// the float4s of a node within a warp are summed by a fixed shuffle tree)
// and adds one partial per warp segment of 32 float4 to the FP64 time
// accumulator hacc[i][segment] (GB300's FP64 rate is a small fraction of
// its FP32 rate: one FP64 add per node and step), then stores r = a dt/C
// and tp = a - (R+S) r.
template <int D>
__global__ void k_flux_adj_p(int64_t n, int64_t m, int ld4, const int64_t* __restrict__ nc_ptr,
                             const int32_t* __restrict__ nc_cell, const float* __restrict__ w,
                             const float2* __restrict__ coef, const float4* __restrict__ Qt,
                             float4* __restrict__ tp, float4* __restrict__ rr, Slots sl,
                             double* __restrict__ hacc, const int32_t* __restrict__ rec_ptr,
                             const int32_t* __restrict__ rec_shot,
                             const int32_t* __restrict__ rec_trace,
                             const float* __restrict__ W, int nt, StepRef sr, float dt) {
  pdl_sync();
  const int l = step_of(sr);
  const bool first = l == nt - 1;
  const float4* __restrict__ p0 = slot_of(sl, l);   // p_l; p_{l+1} in the next slot
  const float4* __restrict__ p1 = p0 + sl.ns4;
  const int64_t total = n * ld4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ld4;
    const int c4 = (int)(t - i * ld4);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!first) {
      float4 bt = a;
      for (int64_t s = __ldg(nc_ptr + i); s < __ldg(nc_ptr + i + 1); ++s) {
        const int64_t e = __ldg(nc_cell + s);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float wk = __ldg(w + s * D + k);
          const float4 qv = __ldg(Qt + ((int64_t)k * m + e) * ld4 + c4);
          bt.x = fmaf(wk, qv.x, bt.x);
          bt.y = fmaf(wk, qv.y, bt.y);
          bt.z = fmaf(wk, qv.z, bt.z);
          bt.w = fmaf(wk, qv.w, bt.w);
        }
      }
      const float4 tv = tp[t];
      a = make_float4(fmaf(dt, bt.x, tv.x), fmaf(dt, bt.y, tv.y), fmaf(dt, bt.z, tv.z),
                      fmaf(dt, bt.w, tv.w));
    }
    const int r0 = __ldg(rec_ptr + i), r1 = __ldg(rec_ptr + i + 1);
    for (int r = r0; r < r1; ++r) {
      const int d = __ldg(rec_shot + r) - 4 * c4;
      if (d < 0 || d > 3) continue;
      const float v = __ldg(W + (int64_t)__ldg(rec_trace + r) * nt + l);
      if (d == 0) a.x += v;
      if (d == 1) a.y += v;
      if (d == 2) a.z += v;
      if (d == 3) a.w += v;
    }
    const float4 x1 = __ldg(p1 + t), x0 = __ldg(p0 + t);
    float h = a.x * (x1.x - x0.x);
    h = fmaf(a.y, x1.y - x0.y, h);
    h = fmaf(a.z, x1.z - x0.z, h);
    h = fmaf(a.w, x1.w - x0.w, h);
    // ld4 is a power of two or a multiple of 32, and t mod 32 is the lane:
    // the gw lanes of a node's segment are active together
    const int gw = ld4 < 32 ? ld4 : 32;
    const int lane = threadIdx.x & 31;
    const unsigned gmask =
        gw == 32 ? 0xffffffffu : (((1u << gw) - 1u) << (lane & ~(gw - 1)));
    for (int off = gw / 2; off > 0; off >>= 1) h += __shfl_xor_sync(gmask, h, off);
    if ((c4 & (gw - 1)) == 0) {
      const int nseg = ld4 < 32 ? 1 : ld4 / 32;
      hacc[i * nseg + c4 / 32] += (double)h;
    }
    const float2 c = __ldg(coef + i);
    const float4 r = make_float4(a.x * c.x, a.y * c.x, a.z * c.x, a.w * c.x);
    rr[t] = r;
    tp[t] = make_float4(fmaf(-c.y, r.x, a.x), fmaf(-c.y, r.y, a.y), fmaf(-c.y, r.z, a.z),
                        fmaf(-c.y, r.w, a.w));
  }
}

// Adjoint cell kernel: Qt^(k) <- (1 - dt zeta_k) Qt^(k) - sum_a dphi_a/dx_k r[v_a]
template <int D>
__global__ void k_flux_adj_q(int64_t m, int ld4, const int32_t* __restrict__ cells,
                             const float* __restrict__ grad, const float* __restrict__ damp,
                             const float4* __restrict__ rr, float4* __restrict__ Qt, float dt) {
  pdl_sync();
  const int64_t total = m * ld4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / ld4;
    const int c4 = (int)(t - e * ld4);
    float4 rv[D + 1];
#pragma unroll
    for (int a = 0; a <= D; ++a)
      rv[a] = __ldg(rr + (int64_t)__ldg(cells + e * (D + 1) + a) * ld4 + c4);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int a = 0; a <= D; ++a) {
        const float g = __ldg(grad + (e * (D + 1) + a) * D + k);
        acc.x = fmaf(g, rv[a].x, acc.x);
        acc.y = fmaf(g, rv[a].y, acc.y);
        acc.z = fmaf(g, rv[a].z, acc.z);
        acc.w = fmaf(g, rv[a].w, acc.w);
      }
      const float keep = 1.0f - dt * __ldg(damp + e * D + k);
      float4* qp = Qt + ((int64_t)k * m + e) * ld4 + c4;
      const float4 o = *qp;
      *qp = make_float4(fmaf(keep, o.x, -acc.x), fmaf(keep, o.y, -acc.y),
                        fmaf(keep, o.z, -acc.z), fmaf(keep, o.w, -acc.w));
    }
  }
}

// gC_i = -sum_seg hacc[i][seg] / C_i (fixed order over the shot segments)
__global__ void k_flux_hsum(int64_t n, int nseg, const double* __restrict__ hacc,
                            const double* __restrict__ C, double* __restrict__ gC) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = 0; j < nseg; ++j) s += hacc[i * nseg + j];
  gC[i] = -s / C[i];
}

// g_e = |e| / (d+1) sum_a gC[v_a]
__global__ void k_flux_cell_grad(int64_t m, int k1, const int32_t* __restrict__ cells,
                                 const double* __restrict__ vol, const double* __restrict__ gC,
                                 double* __restrict__ g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  double s = 0.0;
  for (int a = 0; a < k1; ++a) s += gC[cells[e * k1 + a]];
  g[e] = vol[e] / k1 * s;
}

struct Scratch {
  cudaStream_t st;
  std::vector<void*> p;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (void* x : p) cudaFreeAsync(x, st);
  }
  template <class T>
  T* put(const std::vector<T>& v) {
    void* x = nullptr;
    if (cudaMallocAsync(&x, std::max<size_t>(v.size(), 1) * sizeof(T), st) != cudaSuccess)
      return nullptr;
    p.push_back(x);
    if (!v.empty() &&
        cudaMemcpyAsync(x, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return nullptr;
    return static_cast<T*>(x);
  }
  template <class T>
  T* put(const T* src, size_t count) {  // host array
    return put(std::vector<T>(src, src + count));
  }
  template <class T>
  T* get(size_t count) {
    void* x = nullptr;
    if (cudaMallocAsync(&x, std::max<size_t>(count, 1) * sizeof(T), st) != cudaSuccess)
      return nullptr;
    p.push_back(x);
    return static_cast<T*>(x);
  }
};

// Launch of a step kernel as a programmatic dependent (see pdl_sync).
template <class... KArgs, class... Args>
void launch_pdl(void (*kern)(KArgs...), int grid, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

int grid_for(int64_t total) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
}

// Everything the three entry points share: geometry, layer damping, event
// lists, source amplitudes, per-node coefficients, device inputs.
struct Flux {
  int d = 0, k1 = 0, S = 0, ld = 0, ld4 = 0, nt = 0;
  int64_t n = 0, m = 0, R = 0;
  double dt = 0.0;
  bool host = false;
  cudaStream_t st = nullptr;
  MeshView V;
  CoefArgs c;
  const double* eps_d = nullptr;
  int32_t* cells = nullptr;
  float *grad = nullptr, *w = nullptr, *damp = nullptr;
  int32_t *sp = nullptr, *ss = nullptr, *rp = nullptr, *rs = nullptr, *rt = nullptr;
  float* fl = nullptr;      // f_l (FP32) per step, device
  float2* coef = nullptr;

  // flux update from p (or, with sl.seg, from the slot of step sr)
  void step_q(float* p, float* q, cudaStream_t s, StepRef sr = {0, nullptr},
              Slots sl = {nullptr, 0, 1}) const {
    const int g = grid_for(m * ld4);
    if (d == 2)
      launch_pdl(k_flux_q<2>, g, s, m, ld4, cells, grad, damp,
                 reinterpret_cast<const float4*>(p), reinterpret_cast<float4*>(q), (float)dt, sr,
                 sl);
    else
      launch_pdl(k_flux_q<3>, g, s, m, ld4, cells, grad, damp,
                 reinterpret_cast<const float4*>(p), reinterpret_cast<float4*>(q), (float)dt, sr,
                 sl);
  }
  // node update of step sr: p_{l+1} into pout (nullptr: in place over p),
  // or with sl.seg from the step's slot into the next one
  void step_p(const float* q, float* p, float* traces, StepRef sr, cudaStream_t s,
              float* pout = nullptr, Slots sl = {nullptr, 0, 1}) const {
    const int g = grid_for(n * ld4);
    float4* po = reinterpret_cast<float4*>(pout ? pout : p);
    if (d == 2)
      launch_pdl(k_flux_p<2>, g, s, n, m, ld4, c.nc_ptr, c.nc_cell, w, coef,
                 reinterpret_cast<const float4*>(q), reinterpret_cast<const float4*>(p), po, sp,
                 ss, rp, rs, rt, fl, traces, nt, sr, sl);
    else
      launch_pdl(k_flux_p<3>, g, s, n, m, ld4, c.nc_ptr, c.nc_cell, w, coef,
                 reinterpret_cast<const float4*>(q), reinterpret_cast<const float4*>(p), po, sp,
                 ss, rp, rs, rt, fl, traces, nt, sr, sl);
  }
};

// One captured chunk of steps, replayed with cudaGraphLaunch on the
// caller's stream.  Recorded on a private stream (the caller's may be the
// legacy default stream, which cannot be captured); destroyed with the
// call, after the stream it ran on has drained.
struct Chunk {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t used = nullptr;
  Chunk() = default;
  Chunk(const Chunk&) = delete;
  Chunk& operator=(const Chunk&) = delete;
  ~Chunk() {
    if (!exec) return;
    if (used) cudaStreamSynchronize(used);
    cudaGraphExecDestroy(exec);
  }
  template <class Body>
  int record(Body&& body) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MG_ERR_CUDA;
    int rc = MG_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = MG_ERR_CUDA;
    } else {
      rc = body(cs);
      if (cudaStreamEndCapture(cs, &g) != cudaSuccess && rc == MG_OK) rc = MG_ERR_CUDA;
    }
    if (rc == MG_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
      exec = nullptr;
      rc = MG_ERR_CUDA;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != MG_OK) cudaGetLastError();
    return rc;
  }
  int launch(cudaStream_t st) {
    used = st;
    return cudaGraphLaunch(exec, st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
  }
};

int flux_setup(mg_mesh* M, const double* eps, const mg_shots* shots, const double* wavelet,
               double dt, int nt, const double* xi, const double* zeta, int flags,
               cudaStream_t st, Scratch& X, Flux& F) {
  if (!M || !eps || !shots || !wavelet || nt < 1 || !(dt > 0.0)) return MG_ERR_ARG;
  const HostMesh* hm = host_mesh(M);
  const int d = hm->dim, k1 = d + 1;
  if (d < 2 || d > kMaxDim) return MG_ERR_UNSUPPORTED;
  const int S = shots->n_shots;
  if (S < 1 || !shots->src || !shots->rec_ptr || (shots->rec_ptr[S] > 0 && !shots->rec) ||
      shots->rec_ptr[0] != 0)
    return MG_ERR_ARG;
  const int64_t n = hm->n, m = hm->m, R = shots->rec_ptr[S];
  for (int s = 0; s < S; ++s) {
    if (shots->src[s] < 0 || shots->src[s] >= n || shots->rec_ptr[s + 1] < shots->rec_ptr[s])
      return MG_ERR_ARG;
  }
  for (int64_t r = 0; r < R; ++r)
    if (shots->rec[r] < 0 || shots->rec[r] >= n) return MG_ERR_ARG;
  const bool host = flags & MG_HOST_PTRS;
  F.d = d;
  F.k1 = k1;
  F.S = S;
  F.n = n;
  F.m = m;
  F.R = R;
  F.nt = nt;
  F.dt = dt;
  F.host = host;
  F.st = st;

  // per cell: gradients of the barycentric functions (FP64 -> FP32) and
  // per node-cell incidence: |e| dphi_i/dx_k
  std::vector<float> grad((size_t)m * k1 * d);
  for (int64_t e = 0; e < m; ++e) {
    const int32_t* v = hm->cells.data() + (size_t)e * k1;
    double E[kMaxDim][kMaxDim], inv[kMaxDim][kMaxDim];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b)
        E[a][b] = hm->coords[(size_t)v[b + 1] * d + a] - hm->coords[(size_t)v[0] * d + a];
    // inverse of E (columns x_b - x_0); rows of inv are grad phi_1..phi_d
    double det;
    if (d == 2) {
      det = E[0][0] * E[1][1] - E[0][1] * E[1][0];
      inv[0][0] = E[1][1] / det; inv[0][1] = -E[0][1] / det;
      inv[1][0] = -E[1][0] / det; inv[1][1] = E[0][0] / det;
    } else {
      det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
            E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
            E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const int a1 = (b + 1) % 3, a2 = (b + 2) % 3, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
          inv[a][b] = (E[a1][b1] * E[a2][b2] - E[a1][b2] * E[a2][b1]) / det;
        }
    }
    if (!(det != 0.0) || !std::isfinite(det)) return MG_ERR_ARG;
    for (int k = 0; k < d; ++k) {
      double g0 = 0.0;
      for (int a = 1; a <= d; ++a) {
        const double g = inv[a - 1][k];
        grad[((size_t)e * k1 + a) * d + k] = (float)g;
        g0 -= g;
      }
      grad[((size_t)e * k1) * d + k] = (float)g0;
    }
  }
  std::vector<float> wnc(hm->nc_cell.size() * d);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t s = hm->nc_ptr[i]; s < hm->nc_ptr[i + 1]; ++s) {
      const int32_t e = hm->nc_cell[s];
      int a = 0;
      while (a < k1 && hm->cells[(size_t)e * k1 + a] != i) ++a;
      if (a == k1) return MG_ERR_ARG;
      for (int k = 0; k < d; ++k)
        wnc[(size_t)s * d + k] = (float)(hm->cell_vol[e] * grad[((size_t)e * k1 + a) * d + k]);
    }
  // damping zeta per cell and direction (FP32), sources / receivers per row
  std::vector<float> damp((size_t)m * d, 0.0f);
  if (zeta) {
    std::vector<double> zeta_h((size_t)m * d);
    if (host) std::copy(zeta, zeta + (size_t)m * d, zeta_h.begin());
    else if (cudaMemcpy(zeta_h.data(), zeta, zeta_h.size() * sizeof(double),
                        cudaMemcpyDeviceToHost) != cudaSuccess)
      return MG_ERR_CUDA;
    for (size_t q = 0; q < zeta_h.size(); ++q) {
      if (!(zeta_h[q] >= 0.0) || !std::isfinite(zeta_h[q])) return MG_ERR_ARG;
      damp[q] = (float)zeta_h[q];
    }
  }
  F.ld = S <= 4 ? 4 : ((S + 3) / 4) * 4;
  F.ld4 = F.ld / 4;
  std::vector<int32_t> sp(n + 1, 0), ss(S), rp(n + 1, 0), rs(R), rt(R);
  const std::vector<int32_t>& perm = hm->perm;
  for (int s = 0; s < S; ++s) sp[perm[shots->src[s]] + 1]++;
  for (int64_t r = 0; r < R; ++r) rp[perm[shots->rec[r]] + 1]++;
  for (int64_t i = 0; i < n; ++i) {
    sp[i + 1] += sp[i];
    rp[i + 1] += rp[i];
  }
  {
    std::vector<int32_t> fs(sp.begin(), sp.end() - 1), fr(rp.begin(), rp.end() - 1);
    for (int s = 0; s < S; ++s) ss[fs[perm[shots->src[s]]]++] = s;
    for (int s = 0; s < S; ++s)
      for (int64_t r = shots->rec_ptr[s]; r < shots->rec_ptr[s + 1]; ++r) {
        const int32_t row = perm[shots->rec[r]];
        rs[fr[row]] = s;
        rt[fr[row]++] = (int32_t)r;
      }
  }
  // source amplitudes f_l = dt sum_{m <= l} s_m (FP64 sum, FP32 value)
  std::vector<double> wav_h(nt);
  if (host) std::copy(wavelet, wavelet + nt, wav_h.begin());
  else if (cudaMemcpy(wav_h.data(), wavelet, nt * sizeof(double), cudaMemcpyDeviceToHost) !=
           cudaSuccess)
    return MG_ERR_CUDA;
  std::vector<float> fl_h(nt);
  double acc = 0.0;
  for (int l = 0; l < nt; ++l) {
    acc += dt * wav_h[l];
    fl_h[l] = (float)acc;
  }

  if (mesh_view(M, &F.V) != MG_OK) return MG_ERR_ARG;
  F.eps_d = eps;
  const double* xi_d = xi;
  if (host) {
    F.eps_d = X.put(eps, (size_t)m);
    if (xi) xi_d = X.put(xi, (size_t)m);
    if (!F.eps_d || (xi && !xi_d)) return MG_ERR_OOM;
  }
  if (!(flags & MG_ALLOW_CFL)) {
    double dtc = 0.0;
    const int rc = mg_cfl_dt(M, F.eps_d, 0, st, &dtc);
    if (rc) return rc;
    if (dt > dtc * (1.0 + 1e-12)) return MG_ERR_CFL;
  }
  F.cells = X.put(hm->cells);
  F.grad = X.put(grad);
  F.w = X.put(wnc);
  F.damp = X.put(damp);
  F.sp = X.put(sp);
  F.ss = X.put(ss);
  F.rp = X.put(rp);
  F.rs = X.put(rs);
  F.rt = X.put(rt);
  F.fl = X.put(fl_h);
  F.coef = X.get<float2>(n);
  if (!F.cells || !F.grad || !F.w || !F.damp || !F.sp || !F.ss || !F.rp || !F.rs || !F.rt ||
      !F.fl || !F.coef)
    return MG_ERR_OOM;
  F.c = F.V.coef_base;
  F.c.eps = F.eps_d;
  k_flux_coefs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F.c, xi_d, dt, F.coef);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

struct DeviceScope {
  int prev = 0;
  bool ok = false;
  explicit DeviceScope(int dev) {
    ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() { cudaSetDevice(prev); }
};

#define MG_FX(x)                  \
  do {                            \
    const int rc_ = (x);          \
    if (rc_ != MG_OK) return rc_; \
  } while (0)

// Steps per CUDA-graph chunk for a call (0: plain launches): the handle's
// chunk length, unless MG_NO_GRAPH.
int chunk_len(const mg_mesh* M, int flags) {
  const int c = mesh_graph_chunk(M);
  return (flags & MG_NO_GRAPH) || c < 2 ? 0 : c;
}

}  // namespace
}  // namespace mg

extern "C" int mg_forward_pml(mg_mesh* M, const double* eps, const mg_shots* shots,
                              const double* wavelet, double dt, int nt, const double* xi,
                              const double* zeta, float* traces, void* stream, int flags) {
  using namespace mg;
  if (!M || !eps || !shots || !wavelet || !traces || nt < 1 || !(dt > 0.0)) return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL | MG_NO_GRAPH)) return MG_ERR_UNSUPPORTED;
  DeviceScope scope(mesh_device(M));
  if (!scope.ok) return MG_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch X(st);
  Flux F;
  MG_FX(flux_setup(M, eps, shots, wavelet, dt, nt, xi, zeta, flags, st, X, F));
  const int64_t n = F.n, m = F.m, R = F.R;
  float* p = X.get<float>((size_t)n * F.ld);
  float* q = X.get<float>((size_t)F.d * m * F.ld);
  float* tr = F.host ? X.get<float>((size_t)R * nt) : traces;
  int* base = X.get<int>(1);
  if (!p || !q || !tr || !base) return MG_ERR_OOM;
  if (cudaMemsetAsync(p, 0, (size_t)n * F.ld * sizeof(float), st) ||
      cudaMemsetAsync(q, 0, (size_t)F.d * m * F.ld * sizeof(float), st))
    return MG_ERR_CUDA;
  const int C = chunk_len(M, flags);
  int l = 0;
  Chunk ch;
  if (C && nt >= C) {   // whole chunks: one graph launch each
    MG_FX(launch_set_int(base, 0, st));
    MG_FX(ch.record([&](cudaStream_t cs) {
      for (int j = 0; j < C; ++j) {
        F.step_q(p, q, cs);
        F.step_p(q, p, tr, {j, base}, cs);
      }
      return launch_add_int(base, C, cs);
    }));
    for (; l + C <= nt; l += C) MG_FX(ch.launch(st));
  }
  for (; l < nt; ++l) {
    F.step_q(p, q, st);
    F.step_p(q, p, tr, {l, nullptr}, st);
  }
  if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
  add_launches(M, 1 + 2 * (int64_t)nt);
  if (F.host && cudaMemcpyAsync(traces, tr, (size_t)R * nt * sizeof(float),
                                cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MG_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

extern "C" int mg_jacobian_apply_pml(mg_mesh* M, int level, const double* eps,
                                     const mg_shots* shots, const double* wavelet, double dt,
                                     int nt, const double* xi, const double* zeta,
                                     const double* v, float* jv, void* stream, int flags) {
  using namespace mg;
  if (!M || !eps || !shots || !wavelet || !v || !jv || nt < 1 || !(dt > 0.0)) return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL | MG_NO_GRAPH)) return MG_ERR_UNSUPPORTED;
  const HostMesh* hm = host_mesh(M);
  if (level < 0 || level >= hm->n_levels) return MG_ERR_ARG;
  DeviceScope scope(mesh_device(M));
  if (!scope.ok) return MG_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch X(st);
  Flux F;
  MG_FX(flux_setup(M, eps, shots, wavelet, dt, nt, xi, zeta, flags, st, X, F));
  const int64_t n = F.n, m = F.m, R = F.R, nc = hm->n_cells_level[level];
  const double* v_d = F.host ? X.put(v, (size_t)nc) : v;
  const int32_t* anc = X.put(hm->ancestors[level]);
  double* dv = X.get<double>(m);
  double* C = X.get<double>(n);
  double* dC = X.get<double>(n);
  float* ratio = X.get<float>(n);
  const size_t ns = (size_t)n * F.ld, qs = (size_t)F.d * m * F.ld;
  float* p = X.get<float>(ns);
  float* dp = X.get<float>(ns);
  float* q = X.get<float>(qs);
  float* dq = X.get<float>(qs);
  float* tr = F.host ? X.get<float>((size_t)R * nt) : jv;
  int* base = X.get<int>(1);
  if (!v_d || !anc || !dv || !C || !dC || !ratio || !p || !dp || !q || !dq || !tr || !base)
    return MG_ERR_OOM;
  MG_FX(launch_prolong(m, anc, v_d, nullptr, dv, st));
  const unsigned gn = (unsigned)((n + 255) / 256);
  k_flux_mass<<<gn, 256, 0, st>>>(F.c, F.eps_d, C);
  k_flux_mass<<<gn, 256, 0, st>>>(F.c, dv, dC);
  k_flux_ratio<<<gn, 256, 0, st>>>(n, dC, C, ratio);
  if (cudaMemsetAsync(p, 0, ns * sizeof(float), st) ||
      cudaMemsetAsync(dp, 0, ns * sizeof(float), st) ||
      cudaMemsetAsync(q, 0, qs * sizeof(float), st) ||
      cudaMemsetAsync(dq, 0, qs * sizeof(float), st))
    return MG_ERR_CUDA;
  const int gp = grid_for(n * F.ld4);
  auto step = [&](StepRef sr, cudaStream_t s) {
    F.step_q(p, q, s);
    F.step_q(dp, dq, s);
    if (F.d == 2)
      launch_pdl(k_flux_p_tan<2>, gp, s, n, m, F.ld4, F.c.nc_ptr, F.c.nc_cell, F.w, F.coef,
                 ratio, reinterpret_cast<const float4*>(q), reinterpret_cast<const float4*>(dq),
                 reinterpret_cast<float4*>(p), reinterpret_cast<float4*>(dp), F.sp, F.ss, F.rp,
                 F.rs, F.rt, F.fl, tr, nt, sr);
    else
      launch_pdl(k_flux_p_tan<3>, gp, s, n, m, F.ld4, F.c.nc_ptr, F.c.nc_cell, F.w, F.coef,
                 ratio, reinterpret_cast<const float4*>(q), reinterpret_cast<const float4*>(dq),
                 reinterpret_cast<float4*>(p), reinterpret_cast<float4*>(dp), F.sp, F.ss, F.rp,
                 F.rs, F.rt, F.fl, tr, nt, sr);
  };
  const int CL = chunk_len(M, flags);
  int l = 0;
  Chunk ch;
  if (CL && nt >= CL) {   // whole chunks: one graph launch each
    MG_FX(launch_set_int(base, 0, st));
    MG_FX(ch.record([&](cudaStream_t cs) {
      for (int j = 0; j < CL; ++j) step({j, base}, cs);
      return launch_add_int(base, CL, cs);
    }));
    for (; l + CL <= nt; l += CL) MG_FX(ch.launch(st));
  }
  for (; l < nt; ++l) step({l, nullptr}, st);
  if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
  add_launches(M, 5 + 3 * (int64_t)nt);
  if (F.host && cudaMemcpyAsync(jv, tr, (size_t)R * nt * sizeof(float), cudaMemcpyDeviceToHost,
                                st) != cudaSuccess)
    return MG_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

extern "C" int mg_jacobian_T_apply_pml(mg_mesh* M, int level, const double* eps,
                                       const mg_shots* shots, const double* wavelet, double dt,
                                       int nt, const double* xi, const double* zeta,
                                       const float* w, double* g, int ckpt_every, void* stream,
                                       int flags) {
  using namespace mg;
  if (!M || !eps || !shots || !wavelet || !w || !g || nt < 1 || !(dt > 0.0) || ckpt_every < 1)
    return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL | MG_NO_GRAPH)) return MG_ERR_UNSUPPORTED;
  const HostMesh* hm = host_mesh(M);
  if (level < 0 || level >= hm->n_levels) return MG_ERR_ARG;
  DeviceScope scope(mesh_device(M));
  if (!scope.ok) return MG_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch X(st);
  Flux F;
  MG_FX(flux_setup(M, eps, shots, wavelet, dt, nt, xi, zeta, flags, st, X, F));
  const int64_t n = F.n, m = F.m, R = F.R, nc = hm->n_cells_level[level];
  const int K = std::min(ckpt_every, nt);
  const int nck = (nt + K - 1) / K;
  // one segment (ckpt_every >= nt): the forward keeps every state, and the
  // reverse steps run with no recompute
  const bool keep = nck == 1;
  const size_t ns = (size_t)n * F.ld, qs = (size_t)F.d * m * F.ld;
  const int nseg = F.ld4 < 32 ? 1 : F.ld4 / 32;
  const float* W = F.host ? X.put(w, (size_t)R * nt) : w;
  float* ck_p = X.get<float>(ns * nck);
  float* ck_q = X.get<float>(qs * nck);
  float* seg = X.get<float>(ns * (K + 1));
  float* p = keep ? seg : X.get<float>(ns);   // the forward's state (keep: unused)
  float* q = X.get<float>(qs);
  float* trd = X.get<float>((size_t)R * nt);
  float* tp = X.get<float>(ns);
  float* rr = X.get<float>(ns);
  float* Qt = X.get<float>(qs);
  double* hacc = X.get<double>((size_t)n * nseg);
  double* C = X.get<double>(n);
  double* gC = X.get<double>(n);
  double* vol = X.put(hm->cell_vol);
  double* gf = X.get<double>(m);
  std::vector<int64_t> lp;
  std::vector<int32_t> li;
  level_children(*hm, level, lp, li);
  int64_t* lp_d = X.put(lp);
  int32_t* li_d = X.put(li);
  double* go = F.host ? X.get<double>(nc) : g;
  int* base = X.get<int>(1);
  if (!W || !ck_p || !ck_q || !p || !q || !seg || !trd || !tp || !rr || !Qt || !hacc || !C ||
      !gC || !vol || !gf || !lp_d || !li_d || !go || !base)
    return MG_ERR_OOM;
  if (cudaMemsetAsync(p, 0, ns * sizeof(float), st) ||
      cudaMemsetAsync(q, 0, qs * sizeof(float), st) ||
      cudaMemsetAsync(Qt, 0, qs * sizeof(float), st) ||
      cudaMemsetAsync(hacc, 0, (size_t)n * nseg * sizeof(double), st))
    return MG_ERR_CUDA;
  int64_t launches = 0;
  const int CL = chunk_len(M, flags);
  // p_l in slot l of seg (keep: the whole run, slots 0..nt) or in slot
  // l - l0 of the segment [l0, l0 + K) being reversed
  const Slots sl{reinterpret_cast<float4*>(seg), (int64_t)ns / 4, keep ? nt + 1 : K};
  // forward, keeping (p_l, q_{l-1/2}) at l = 0, K, 2K, ... (or every p_l)
  if (keep && cudaMemsetAsync(seg, 0, ns * sizeof(float), st)) return MG_ERR_CUDA;
  auto fwd_slots = [&](StepRef sr, cudaStream_t s) {   // p_l in its slot, p_{l+1} the next
    F.step_q(seg, q, s, sr, sl);
    F.step_p(q, seg, trd, sr, s, nullptr, sl);
  };
  auto fwd = [&](StepRef sr, cudaStream_t s) {
    if (keep) {
      fwd_slots(sr, s);
    } else {
      F.step_q(p, q, s);
      F.step_p(q, p, trd, sr, s);
    }
  };
  // graph chunks: keep, CL steps; else one checkpoint interval of K steps
  const int LF = keep ? CL : (CL ? K : 0);
  int l = 0;
  Chunk chf;
  if (LF >= 2 && nt >= LF) {
    MG_FX(launch_set_int(base, 0, st));
    MG_FX(chf.record([&](cudaStream_t cs) {
      for (int j = 0; j < LF; ++j) fwd({j, base}, cs);
      return launch_add_int(base, LF, cs);
    }));
    for (; l + LF <= nt; l += LF) {
      if (!keep &&
          (cudaMemcpyAsync(ck_p + ns * (l / K), p, ns * sizeof(float), cudaMemcpyDeviceToDevice,
                           st) ||
           cudaMemcpyAsync(ck_q + qs * (l / K), q, qs * sizeof(float), cudaMemcpyDeviceToDevice,
                           st)))
        return MG_ERR_CUDA;
      MG_FX(chf.launch(st));
      launches += 2 * LF;
    }
  }
  for (; l < nt; ++l) {
    if (!keep && l % K == 0 &&
        (cudaMemcpyAsync(ck_p + ns * (l / K), p, ns * sizeof(float), cudaMemcpyDeviceToDevice,
                         st) ||
         cudaMemcpyAsync(ck_q + qs * (l / K), q, qs * sizeof(float), cudaMemcpyDeviceToDevice,
                         st)))
      return MG_ERR_CUDA;
    fwd({l, nullptr}, st);
    launches += 2;
  }
  // reverse step l: p_l, p_{l+1} from their slots
  const int gp = grid_for(n * F.ld4), gq = grid_for(m * F.ld4);
  const float fdt = (float)dt;
  auto rev = [&](StepRef sr, cudaStream_t s) {
    if (F.d == 2) {
      launch_pdl(k_flux_adj_p<2>, gp, s, n, m, F.ld4, F.c.nc_ptr, F.c.nc_cell, F.w, F.coef,
                 reinterpret_cast<const float4*>(Qt), reinterpret_cast<float4*>(tp),
                 reinterpret_cast<float4*>(rr), sl, hacc, F.rp, F.rs, F.rt, W, nt, sr, fdt);
      launch_pdl(k_flux_adj_q<2>, gq, s, m, F.ld4, F.cells, F.grad, F.damp,
                 reinterpret_cast<const float4*>(rr), reinterpret_cast<float4*>(Qt), fdt);
    } else {
      launch_pdl(k_flux_adj_p<3>, gp, s, n, m, F.ld4, F.c.nc_ptr, F.c.nc_cell, F.w, F.coef,
                 reinterpret_cast<const float4*>(Qt), reinterpret_cast<float4*>(tp),
                 reinterpret_cast<float4*>(rr), sl, hacc, F.rp, F.rs, F.rt, W, nt, sr, fdt);
      launch_pdl(k_flux_adj_q<3>, gq, s, m, F.ld4, F.cells, F.grad, F.damp,
                 reinterpret_cast<const float4*>(rr), reinterpret_cast<float4*>(Qt), fdt);
    }
  };
  // segment [l0, l0 + len) with p_{l0} in slot 0 and q_{l0-1/2} in q: its
  // forward steps into slots 1..len (q in place), then the reverse steps
  // l0 + len - 1 .. l0; s0 is step l0
  auto segment = [&](int len, StepRef s0, cudaStream_t s) {
    for (int j = 0; j < len; ++j) fwd_slots({s0.l + j, s0.base}, s);
    for (int j = len - 1; j >= 0; --j) rev({s0.l + j, s0.base}, s);
  };
  Chunk chr;
  if (keep) {   // reverse steps nt-1 .. 0 in chunks of CL (base: the chunk's first step)
    int k = nt;   // steps below k remain
    if (CL >= 2 && nt >= CL) {
      MG_FX(launch_set_int(base, nt - 1, st));
      MG_FX(chr.record([&](cudaStream_t cs) {
        for (int j = 0; j < CL; ++j) rev({-j, base}, cs);
        return launch_add_int(base, -CL, cs);
      }));
      for (; k >= CL; k -= CL) {
        MG_FX(chr.launch(st));
        launches += 2 * CL;
      }
    }
    for (int r = k - 1; r >= 0; --r) {
      rev({r, nullptr}, st);
      launches += 2;
    }
  } else {
    const int nfull = nt / K;
    auto load = [&](int c) {   // checkpoint c into slot 0 and q
      return cudaMemcpyAsync(seg, ck_p + ns * c, ns * sizeof(float), cudaMemcpyDeviceToDevice,
                             st) == cudaSuccess &&
             cudaMemcpyAsync(q, ck_q + qs * c, qs * sizeof(float), cudaMemcpyDeviceToDevice,
                             st) == cudaSuccess;
    };
    if (nt % K) {   // the last, shorter segment: plain launches
      if (!load(nfull)) return MG_ERR_CUDA;
      segment(nt - nfull * K, {nfull * K, nullptr}, st);
      launches += 4 * (int64_t)(nt - nfull * K);
    }
    if (CL && K >= 2 && nfull >= 1) {   // full segments: one graph launch each
      MG_FX(launch_set_int(base, (nfull - 1) * K, st));
      MG_FX(chr.record([&](cudaStream_t cs) {
        segment(K, {0, base}, cs);
        return launch_add_int(base, -K, cs);
      }));
      for (int c = nfull - 1; c >= 0; --c) {
        if (!load(c)) return MG_ERR_CUDA;
        MG_FX(chr.launch(st));
        launches += 4 * (int64_t)K;
      }
    } else {
      for (int c = nfull - 1; c >= 0; --c) {
        if (!load(c)) return MG_ERR_CUDA;
        segment(K, {c * K, nullptr}, st);
        launches += 4 * (int64_t)K;
      }
    }
  }
  // gradient: C-sensitivity per node, per finest cell, restricted to the level
  const unsigned gn = (unsigned)((n + 255) / 256), gm = (unsigned)((m + 255) / 256);
  k_flux_mass<<<gn, 256, 0, st>>>(F.c, F.eps_d, C);
  k_flux_hsum<<<gn, 256, 0, st>>>(n, nseg, hacc, C, gC);
  k_flux_cell_grad<<<gm, 256, 0, st>>>(m, F.k1, F.cells, vol, gC, gf);
  if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
  MG_FX(launch_restrict(nc, lp_d, li_d, gf, go, st));
  add_launches(M, launches + 5);
  if (F.host && cudaMemcpyAsync(g, go, nc * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess)
    return MG_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}
