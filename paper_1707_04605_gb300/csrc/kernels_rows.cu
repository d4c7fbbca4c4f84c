// Row-parallel (untiled) leapfrog kernels: forward step, forward+tangent
// step and reverse adjoint step, for every shot of a batch.
//
// State layout: node-major [row][ld] FP32, ld = padded shot count.  A lane
// carries NV float4 (4*NV shots); LPR lanes cover a source tile of
// TW = 4*NV*LPR shots of one row, so a warp advances 32/LPR rows.  The
// lane's j-th float4 holds shots base + 4*LPR*j .. +3, so every vector load
// of the LPR lanes of a row reads one contiguous 16*LPR-byte span.
// The stiffness entry (col, K) of a row is loaded once per lane and serves
// all 4*NV shots of the lane; the NV gathers of a neighbour are independent
// and in flight together.
#include <cuda_runtime.h>

#include "../../include/mgwave.h"
#include "device_util.cuh"
#include "kernels.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

using namespace dev;

struct Row {
  const int2* e;  // entry 0 of the row (stride kSliceH)
  int w;          // entries of the row's slice, diagonal first
};

__device__ __forceinline__ Row row_of(const DevEll& K, int row) {
  const int slice = row / kSliceH;
  Row r;
  r.e = K.ell + __ldg(K.slice_off + slice) + (row - slice * kSliceH);
  r.w = __ldg(K.slice_w + slice);
  return r;
}

// acc[j] = sum_k K_k x[col_k][lane's float4 j], self[j] = x[row][...].
template <int LPR, int NV>
__device__ __forceinline__ void row_sum(const Row& r, const float* __restrict__ xb, int row,
                                        int ld, float4 (&self)[NV], float4 (&acc)[NV]) {
  const float* xr = xb + (size_t)row * ld;
#pragma unroll
  for (int j = 0; j < NV; ++j) self[j] = __ldg(reinterpret_cast<const float4*>(xr + 4 * LPR * j));
  const float v0 = __int_as_float(__ldg(r.e).y);
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = scale4(v0, self[j]);
#pragma unroll 2
  for (int k = 1; k < r.w; ++k) {
    const int2 ek = __ldg(r.e + k * kSliceH);
    const float v = __int_as_float(ek.y);
    const float* xc = xb + (size_t)ek.x * ld;
    float4 x[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) x[j] = __ldg(reinterpret_cast<const float4*>(xc + 4 * LPR * j));
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = fma4(v, x[j], acc[j]);
  }
}

template <int LPR, int NV>
__device__ __forceinline__ void row_sum2(const Row& r, const float* __restrict__ pb,
                                         const float* __restrict__ qb, int row, int ld,
                                         float4 (&ps)[NV], float4 (&qs)[NV], float4 (&pacc)[NV],
                                         float4 (&qacc)[NV]) {
  const size_t ro = (size_t)row * ld;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    ps[j] = __ldg(reinterpret_cast<const float4*>(pb + ro + 4 * LPR * j));
    qs[j] = __ldg(reinterpret_cast<const float4*>(qb + ro + 4 * LPR * j));
  }
  const float v0 = __int_as_float(__ldg(r.e).y);
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    pacc[j] = scale4(v0, ps[j]);
    qacc[j] = scale4(v0, qs[j]);
  }
#pragma unroll 2
  for (int k = 1; k < r.w; ++k) {
    const int2 ek = __ldg(r.e + k * kSliceH);
    const float v = __int_as_float(ek.y);
    const size_t o = (size_t)ek.x * ld;
    float4 x[NV], y[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      x[j] = __ldg(reinterpret_cast<const float4*>(pb + o + 4 * LPR * j));
      y[j] = __ldg(reinterpret_cast<const float4*>(qb + o + 4 * LPR * j));
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      pacc[j] = fma4(v, x[j], pacc[j]);
      qacc[j] = fma4(v, y[j], qacc[j]);
    }
  }
}

// Shot `s` of the batch as (float4 index j, component d) of this lane, or
// j = -1 when another lane (or another source tile) owns it.
template <int LPR, int NV>
__device__ __forceinline__ int owner(int s, int tile0, int lr, int& d) {
  const int rel = s - tile0;
  if (rel < 0 || rel >= 4 * LPR * NV) return -1;
  const int within = rel % (4 * LPR);
  if (within / 4 != lr) return -1;
  d = within % 4;
  return rel / (4 * LPR);
}

template <int NV>
__device__ __forceinline__ void add_to(float4 (&v)[NV], int j, int d, float x) {
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i == j) add_comp(v[i], d, x);
}

template <int NV>
__device__ __forceinline__ float get_from(const float4 (&v)[NV], int j, int d) {
  float out = 0.0f;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i == j) out = get_comp(v[i], d);
  return out;
}

template <int LPR, int NV>
__global__ void __launch_bounds__(kThreads) k_step_rows(StepArgs a) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blockIdx.x * kWarps + warp) * RPW + lane / LPR;
  if (row >= a.K.n) return;
  const int lr = lane % LPR;
  const int tile0 = blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  const Row r = row_of(a.K, row);
  const float4 c = __ldg(a.coef + row);
  const size_t ro = (size_t)row * a.ld + base;
  float4 old[NV], self[NV], acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) old[j] = *reinterpret_cast<const float4*>(a.pm + ro + 4 * LPR * j);
  row_sum<LPR, NV>(r, a.p + base, row, a.ld, self, acc);
  float4 out[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = leap(c, self[j], old[j], acc[j]);
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  const int s0 = __ldg(a.ev.src_ptr + row), s1 = __ldg(a.ev.src_ptr + row + 1);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.ev.src_shot + q), tile0, lr, d);
      if (j >= 0) add_to<NV>(out, j, d, sv);
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) st4(a.pout + ro + 4 * LPR * j, out[j]);
  if (a.traces) {
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.ev.rec_shot + q), tile0, lr, d);
      if (j >= 0) a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = get_from<NV>(out, j, d);
    }
  }
}

template <int LPR, int NV>
__global__ void __launch_bounds__(kThreads) k_tangent_rows(TangentArgs a) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blockIdx.x * kWarps + warp) * RPW + lane / LPR;
  if (row >= a.f.K.n) return;
  const int lr = lane % LPR;
  const int tile0 = blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  const int ld = a.f.ld;
  const Row r = row_of(a.f.K, row);
  const float4 c = __ldg(a.f.coef + row);
  const float2 tc = __ldg(a.tcoef + row);
  const size_t ro = (size_t)row * ld + base;
  float4 pold[NV], qold[NV], ps[NV], qs[NV], pacc[NV], qacc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    pold[j] = *reinterpret_cast<const float4*>(a.f.pm + ro + 4 * LPR * j);
    qold[j] = *reinterpret_cast<const float4*>(a.qm + ro + 4 * LPR * j);
  }
  row_sum2<LPR, NV>(r, a.f.p + base, a.q + base, row, ld, ps, qs, pacc, qacc);
  float4 pn[NV], qn[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) pn[j] = leap(c, ps[j], pold[j], pacc[j]);
  const int l = a.f.step + (a.f.step_base ? *a.f.step_base : 0);
  const int s0 = __ldg(a.f.ev.src_ptr + row), s1 = __ldg(a.f.ev.src_ptr + row + 1);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.f.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.f.ev.src_shot + q), tile0, lr, d);
      if (j >= 0) add_to<NV>(pn, j, d, sv);
    }
  }
  // dp+ = alpha dp - beta dp- - gamma K dp - cm (p+ - 2p + p-) - cd (p+ - p-)
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    qn[j] = tangent_fix(leap(c, qs[j], qold[j], qacc[j]), pn[j], ps[j], pold[j], tc);
    st4(a.f.pout + ro + 4 * LPR * j, pn[j]);
    st4(a.qm + ro + 4 * LPR * j, qn[j]);
  }
  const int r0 = __ldg(a.f.ev.rec_ptr + row), r1 = __ldg(a.f.ev.rec_ptr + row + 1);
  for (int q = r0; q < r1; ++q) {
    int d;
    const int j = owner<LPR, NV>(__ldg(a.f.ev.rec_shot + q), tile0, lr, d);
    if (j >= 0) a.dtraces[(size_t)__ldg(a.f.ev.rec_trace + q) * a.f.nt + l] = get_from<NV>(qn, j, d);
  }
}

template <int LPR, int NV>
__global__ void __launch_bounds__(kThreads) k_adjoint_rows(AdjointArgs a) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blockIdx.x * kWarps + warp) * RPW + lane / LPR;
  const bool valid = row < a.K.n;
  const int lr = lane % LPR;
  const int tile0 = blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  float t1 = 0.0f, t2 = 0.0f;
  if (valid) {
    const Row r = row_of(a.K, row);
    const float4 c = __ldg(a.coef + row);
    const size_t ro = (size_t)row * a.ld + base;
    float4 old[NV], pk[NV], self[NV], acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      old[j] = *reinterpret_cast<const float4*>(a.mu1 + ro + 4 * LPR * j);  // mu_{k+1}
      pk[j] = __ldg(reinterpret_cast<const float4*>(a.pk + ro + 4 * LPR * j));
    }
    row_sum<LPR, NV>(r, a.mu + base, row, a.ld, self, acc);
    float4 out[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = leap(c, self[j], old[j], acc[j]);
    const int k = a.k + (a.step_base ? *a.step_base : 0);
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.ev.rec_shot + q), tile0, lr, d);
      if (j >= 0)
        add_to<NV>(out, j, d, c.w * __ldg(a.w + (size_t)__ldg(a.ev.rec_trace + q) * a.nt + (k - 1)));
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      st4(a.mu1 + ro + 4 * LPR * j, out[j]);
      adj_terms(pk[j], out[j], self[j], old[j], t1, t2);
    }
  }
#pragma unroll
  for (int off = LPR / 2; off > 0; off >>= 1) {
    t1 += __shfl_xor_sync(0xffffffffu, t1, off);
    t2 += __shfl_xor_sync(0xffffffffu, t2, off);
  }
  if (valid && lr == 0) {
    const size_t gi = (size_t)blockIdx.y * a.K.n + row;
    kahan_add(a.G + gi, a.Gc + gi, t1);
    kahan_add(a.H + gi, a.Hc + gi, t2);
  }
}

// Launch shape for a padded shot count and NV float4 per lane.
struct Shape {
  int lpr, nv;
  dim3 grid;
};

Shape shape_of(int n, int S_pad, int nv) {
  while (nv > 1 && 4 * nv > S_pad) nv >>= 1;
  Shape s;
  s.nv = nv;
  s.lpr = S_pad / (4 * nv) >= 32 ? 32 : S_pad / (4 * nv);
  const int rows_per_block = kWarps * (32 / s.lpr);
  s.grid = dim3((n + rows_per_block - 1) / rows_per_block, S_pad / (4 * nv * s.lpr));
  return s;
}

#define MG_ROWS_SWITCH(KERN, ARGS)                                                         \
  switch (sh.lpr * 8 + sh.nv) {                                                            \
    case 32 * 8 + 1: KERN<32, 1><<<sh.grid, kThreads, 0, st>>>(ARGS); break;               \
    case 32 * 8 + 2: KERN<32, 2><<<sh.grid, kThreads, 0, st>>>(ARGS); break;               \
    case 32 * 8 + 4: KERN<32, 4><<<sh.grid, kThreads, 0, st>>>(ARGS); break;               \
    case 16 * 8 + 1: KERN<16, 1><<<sh.grid, kThreads, 0, st>>>(ARGS); break;               \
    case 16 * 8 + 2: KERN<16, 2><<<sh.grid, kThreads, 0, st>>>(ARGS); break;               \
    case 16 * 8 + 4: KERN<16, 4><<<sh.grid, kThreads, 0, st>>>(ARGS); break;               \
    case 8 * 8 + 1: KERN<8, 1><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 8 * 8 + 2: KERN<8, 2><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 8 * 8 + 4: KERN<8, 4><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 4 * 8 + 1: KERN<4, 1><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 4 * 8 + 2: KERN<4, 2><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 4 * 8 + 4: KERN<4, 4><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 2 * 8 + 1: KERN<2, 1><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 2 * 8 + 2: KERN<2, 2><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 2 * 8 + 4: KERN<2, 4><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 1 * 8 + 1: KERN<1, 1><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 1 * 8 + 2: KERN<1, 2><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    case 1 * 8 + 4: KERN<1, 4><<<sh.grid, kThreads, 0, st>>>(ARGS); break;                 \
    default: return MG_ERR_ARG;                                                            \
  }

}  // namespace

int rows_tiles(int S_pad, int nv) { return (int)shape_of(1, S_pad, nv).grid.y; }

int launch_step(const StepArgs& a, int S_pad, cudaStream_t st) {
  const Shape sh = shape_of(a.K.n, S_pad, a.batch);
  MG_ROWS_SWITCH(k_step_rows, a)
  return check_launch();
}

int launch_tangent(const TangentArgs& a, int S_pad, cudaStream_t st) {
  const Shape sh = shape_of(a.f.K.n, S_pad, a.f.batch);
  MG_ROWS_SWITCH(k_tangent_rows, a)
  return check_launch();
}

int launch_adjoint(const AdjointArgs& a, int S_pad, cudaStream_t st) {
  const Shape sh = shape_of(a.K.n, S_pad, a.batch);
  MG_ROWS_SWITCH(k_adjoint_rows, a)
  return check_launch();
}
#undef MG_ROWS_SWITCH

}  // namespace mg
