// CUDA kernels of the leapfrog wave path (sm_103a).
//
// State layout: node-major, [row][ld] FP32 with the shots of a batch in the
// fast dimension (ld = padded shot count, a multiple of 4).  A lane owns 4
// consecutive shots (one float4); LPR lanes cover the <=128 shots of a
// source tile of one row, so a warp advances 32/LPR rows.  Neighbour rows
// p[col][tile] are therefore gathered as coalesced 16-byte-per-lane loads,
// and the stiffness entry (col, K) of a row is a warp-uniform (LPR = 32) or
// contiguous (LPR < 32, consecutive rows of one ELL slice) 8-byte load that
// is shared by every shot of the tile.  No tensor cores: the step is a
// sparse product, bound by memory traffic, not a dense contraction.
#include <cuda_runtime.h>

#include "../../include/mgwave.h"
#include "kernels.cuh"
#include "mg_internal.h"
#include "device_util.cuh"

namespace mg {
namespace {

using namespace dev;

// Row prologue: every load that depends only on the row index is issued
// before the first dependent one, so a row costs three memory round trips
// (row data, stiffness entries, neighbour gathers) instead of one per field.
struct RowIn {
  const int2* e;   // first ELL entry of the row (stride kSliceH)
  int w;           // entries in the row's slice (diagonal first)
};

__device__ __forceinline__ RowIn row_in(const DevEll& K, int row) {
  const int slice = row / kSliceH;
  const int rl = row - slice * kSliceH;
  RowIn r;
  r.e = K.ell + __ldg(K.slice_off + slice) + rl;
  r.w = __ldg(K.slice_w + slice);
  return r;
}

// acc += sum_{k=1}^{w-1} K_k p[col_k][src0..src0+3], B entries per batch:
// the batch's B stiffness entries are loaded together, then its B float4
// gathers are all in flight before the first FMA.
template <int B>
__device__ __forceinline__ float4 gather_acc(RowIn r, const float* __restrict__ p, int ld,
                                             int src0, float4 acc) {
  for (int k0 = 1; k0 < r.w; k0 += B) {
    int2 ek[B];
#pragma unroll
    for (int j = 0; j < B; ++j)
      ek[j] = (k0 + j < r.w) ? __ldg(r.e + (k0 + j) * kSliceH) : make_int2(-1, 0);
    float4 x[B];
#pragma unroll
    for (int j = 0; j < B; ++j)
      x[j] = ek[j].x >= 0 ? ld4(p + (size_t)ek[j].x * ld + src0) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < B; ++j) acc = fma4(__int_as_float(ek[j].y), x[j], acc);
  }
  return acc;
}

template <int B>
__device__ __forceinline__ void gather_acc2(RowIn r, const float* __restrict__ p,
                                            const float* __restrict__ q, int ld, int src0,
                                            float4& pacc, float4& qacc) {
  for (int k0 = 1; k0 < r.w; k0 += B) {
    int2 ek[B];
#pragma unroll
    for (int j = 0; j < B; ++j)
      ek[j] = (k0 + j < r.w) ? __ldg(r.e + (k0 + j) * kSliceH) : make_int2(-1, 0);
    float4 x[B], y[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const bool ok = ek[j].x >= 0;
      const size_t o = (size_t)(ok ? ek[j].x : 0) * ld + src0;
      x[j] = ok ? ld4(p + o) : make_float4(0.f, 0.f, 0.f, 0.f);
      y[j] = ok ? ld4(q + o) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) {
      pacc = fma4(__int_as_float(ek[j].y), x[j], pacc);
      qacc = fma4(__int_as_float(ek[j].y), y[j], qacc);
    }
  }
}

template <int LPR, int B>
__global__ void __launch_bounds__(kThreads) k_step(StepArgs a) {
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int row = (blockIdx.x * kWarps + warp) * RPW + lane / LPR;
  if (row >= a.K.n) return;
  const int src0 = blockIdx.y * kTile + (lane % LPR) * 4;
  const size_t ro = (size_t)row * a.ld + src0;
  // round trip 1: row-only data
  const RowIn r = row_in(a.K, row);
  const float4 self = ld4(a.p + ro);
  const float4 old = ld4v(a.pm + ro);
  const float4 c = __ldg(a.coef + row);
  const int s0 = __ldg(a.ev.src_ptr + row), s1 = __ldg(a.ev.src_ptr + row + 1);
  const int r0 = a.traces ? __ldg(a.ev.rec_ptr + row) : 0;
  const int r1 = a.traces ? __ldg(a.ev.rec_ptr + row + 1) : 0;
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  // rounds 2-3: stiffness entries, then neighbour gathers
  float4 acc = scale4(__int_as_float(__ldg(r.e).y), self);
  acc = gather_acc<B>(r, a.p, a.ld, src0, acc);
  float4 out = leap(c, self, old, acc);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      const int d = __ldg(a.ev.src_shot + q) - src0;
      if (d >= 0 && d < 4) add_comp(out, d, sv);
    }
  }
  st4(a.pout + ro, out);
  for (int q = r0; q < r1; ++q) {
    const int d = __ldg(a.ev.rec_shot + q) - src0;
    if (d >= 0 && d < 4)
      a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = get_comp(out, d);
  }
}

// Plain single-shot step (the one-source comparator): one thread per row,
// scalar state, sliced-ELL entries read coalesced across the warp (a warp is
// one slice).
__global__ void __launch_bounds__(256) k_step_single(StepArgs a, int shot) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= a.K.n) return;
  const RowIn r = row_in(a.K, row);
  const float self = __ldg(a.p + row);
  const float old = a.pm[row];
  const float4 c = __ldg(a.coef + row);
  float acc = __int_as_float(__ldg(r.e).y) * self;
  for (int k = 1; k < r.w; ++k) {
    const int2 ek = __ldg(r.e + k * kSliceH);
    acc = fmaf(__int_as_float(ek.y), __ldg(a.p + ek.x), acc);
  }
  float out = c.x * self - c.y * old - c.z * acc;
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  const int s0 = __ldg(a.ev.src_ptr + row), s1 = __ldg(a.ev.src_ptr + row + 1);
  for (int q = s0; q < s1; ++q)
    if (__ldg(a.ev.src_shot + q) == shot) out += c.z * __ldg(a.wavelet + l);
  a.pout[row] = out;
  if (a.traces) {
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q)
      if (__ldg(a.ev.rec_shot + q) == shot)
        a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = out;
  }
}

template <int LPR, int B>
__global__ void __launch_bounds__(kThreads) k_tangent(TangentArgs a) {
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int row = (blockIdx.x * kWarps + warp) * RPW + lane / LPR;
  if (row >= a.f.K.n) return;
  const int src0 = blockIdx.y * kTile + (lane % LPR) * 4;
  const int ld = a.f.ld;
  const size_t ro = (size_t)row * ld + src0;
  const RowIn r = row_in(a.f.K, row);
  const float4 ps = ld4(a.f.p + ro), qs = ld4(a.q + ro);
  const float4 pold = ld4v(a.f.pm + ro), qold = ld4v(a.qm + ro);
  const float4 c = __ldg(a.f.coef + row);
  const float2 tc = __ldg(a.tcoef + row);
  const int s0 = __ldg(a.f.ev.src_ptr + row), s1 = __ldg(a.f.ev.src_ptr + row + 1);
  const int r0 = __ldg(a.f.ev.rec_ptr + row), r1 = __ldg(a.f.ev.rec_ptr + row + 1);
  const int l = a.f.step + (a.f.step_base ? *a.f.step_base : 0);
  const float v0 = __int_as_float(__ldg(r.e).y);
  float4 acc = scale4(v0, ps), qacc = scale4(v0, qs);
  gather_acc2<B>(r, a.f.p, a.q, ld, src0, acc, qacc);
  float4 pn = leap(c, ps, pold, acc);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.f.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      const int d = __ldg(a.f.ev.src_shot + q) - src0;
      if (d >= 0 && d < 4) add_comp(pn, d, sv);
    }
  }
  // dp+ = alpha dp - beta dp- - gamma K dp - cm (p+ - 2p + p-) - cd (p+ - p-)
  float4 qn = leap(c, qs, qold, qacc);
#define MG_TAN(X) qn.X -= tc.x * ((pn.X - 2.0f * ps.X) + pold.X) + tc.y * (pn.X - pold.X);
  MG_TAN(x) MG_TAN(y) MG_TAN(z) MG_TAN(w)
#undef MG_TAN
  st4(a.f.pout + ro, pn);
  st4(a.qm + ro, qn);
  for (int q = r0; q < r1; ++q) {
    const int d = __ldg(a.f.ev.rec_shot + q) - src0;
    if (d >= 0 && d < 4)
      a.dtraces[(size_t)__ldg(a.f.ev.rec_trace + q) * a.f.nt + l] = get_comp(qn, d);
  }
}

template <int LPR, int B>
__global__ void __launch_bounds__(kThreads) k_adjoint(AdjointArgs a) {
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int row = (blockIdx.x * kWarps + warp) * RPW + lane / LPR;
  const bool valid = row < a.K.n;
  const int src0 = blockIdx.y * kTile + (lane % LPR) * 4;
  float t1 = 0.0f, t2 = 0.0f;
  if (valid) {
    const size_t ro = (size_t)row * a.ld + src0;
    const RowIn r = row_in(a.K, row);
    const float4 self = ld4(a.mu + ro);
    const float4 old = ld4v(a.mu1 + ro);  // mu_{k+1}
    const float4 pk = ld4(a.pk + ro);
    const float4 c = __ldg(a.coef + row);
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    const int k = a.k + (a.step_base ? *a.step_base : 0);
    float4 acc = scale4(__int_as_float(__ldg(r.e).y), self);
    acc = gather_acc<B>(r, a.mu, a.ld, src0, acc);
    float4 out = leap(c, self, old, acc);
    for (int q = r0; q < r1; ++q) {
      const int d = __ldg(a.ev.rec_shot + q) - src0;
      if (d >= 0 && d < 4)
        add_comp(out, d, c.w * __ldg(a.w + (size_t)__ldg(a.ev.rec_trace + q) * a.nt + (k - 1)));
    }
    st4(a.mu1 + ro, out);
#define MG_ACC(X)                                                              \
  t1 = fmaf(pk.X, (out.X - 2.0f * self.X) + old.X, t1);                        \
  t2 = fmaf(pk.X, out.X - old.X, t2);
    MG_ACC(x) MG_ACC(y) MG_ACC(z) MG_ACC(w)
#undef MG_ACC
  }
#pragma unroll
  for (int off = LPR / 2; off > 0; off >>= 1) {
    t1 += __shfl_xor_sync(0xffffffffu, t1, off);
    t2 += __shfl_xor_sync(0xffffffffu, t2, off);
  }
  if (valid && (lane % LPR) == 0) {
    const size_t gi = (size_t)blockIdx.y * a.K.n + row;
    kahan_add(a.G + gi, a.Gc + gi, t1);
    kahan_add(a.H + gi, a.Hc + gi, t2);
  }
}

__global__ void k_coefs(CoefArgs a) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n) return;
  double m = 0.0, D = 0.0;
  for (int64_t q = a.nc_ptr[r]; q < a.nc_ptr[r + 1]; ++q) m += a.eps[a.nc_cell[q]] * a.nc_w[q];
  if (a.bc == MG_BC_ABC1)
    for (int64_t q = a.nf_ptr[r]; q < a.nf_ptr[r + 1]; ++q)
      D += sqrt(a.eps[a.nf_cell[q]]) * a.nf_w[q];
  const double w = m + 0.5 * a.dt * D;
  float4 c = make_float4((float)(2.0 * m / w), (float)((m - 0.5 * a.dt * D) / w),
                         (float)(a.dt * a.dt / w), (float)(1.0 / w));
  if (a.bc == MG_BC_DIRICHLET && a.is_bnd[r]) c = make_float4(0.f, 0.f, 0.f, 0.f);
  a.coef[r] = c;
  if (a.mass) a.mass[r] = m;
}

__global__ void k_tangent_coefs(TangentCoefArgs a) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.c.n) return;
  double m = 0.0, D = 0.0, dm = 0.0, dD = 0.0;
  for (int64_t q = a.c.nc_ptr[r]; q < a.c.nc_ptr[r + 1]; ++q) {
    const int e = a.c.nc_cell[q];
    m += a.c.eps[e] * a.c.nc_w[q];
    dm += a.v[a.anc[e]] * a.c.nc_w[q];
  }
  if (a.c.bc == MG_BC_ABC1)
    for (int64_t q = a.c.nf_ptr[r]; q < a.c.nf_ptr[r + 1]; ++q) {
      const int e = a.c.nf_cell[q];
      const double se = sqrt(a.c.eps[e]);
      D += se * a.c.nf_w[q];
      dD += a.v[a.anc[e]] / (2.0 * se) * a.c.nf_w[q];
    }
  const double w = m + 0.5 * a.c.dt * D;
  float2 t = make_float2((float)(dm / w), (float)(a.c.dt * dD / (2.0 * w)));
  if (a.c.bc == MG_BC_DIRICHLET && a.c.is_bnd[r]) t = make_float2(0.f, 0.f);
  a.tcoef[r] = t;
}

// max_i row_abs_i / m_i; positive doubles order like their bit patterns,
// so blocks combine with an integer atomicMax (out zeroed beforehand).
__global__ void k_cfl_reduce(int32_t n, const double* row_abs, const double* mass,
                             unsigned long long* out) {
  __shared__ double sm[256];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  sm[threadIdx.x] = r < n ? row_abs[r] / mass[r] : 0.0;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));
}

__device__ __forceinline__ double total(const float* s, const float* c, int n,
                                        int tiles, int r) {
  double t = 0.0;
  for (int j = 0; j < tiles; ++j) t += (double)s[(size_t)j * n + r] - (double)c[(size_t)j * n + r];
  return t;
}

__global__ void k_cell_gradient(GradArgs a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.m) return;
  double gs = 0.0;
  for (int j = 0; j < a.k; ++j) gs += total(a.G, a.Gc, a.n, a.tiles, a.cells[e * a.k + j]);
  double g = -a.vol[e] / a.k * gs;
  if (a.bc == MG_BC_ABC1) {
    const double se = sqrt(a.eps[e]);
    for (int64_t q = a.cf_ptr[e]; q < a.cf_ptr[e + 1]; ++q) {
      const int f = a.cf_facet[q];
      double hs = 0.0;
      for (int j = 0; j < a.dim; ++j) hs += total(a.H, a.Hc, a.n, a.tiles, a.bnd[(int64_t)f * a.dim + j]);
      g -= 0.5 * a.dt * a.bnd_meas[f] / (2.0 * a.dim * se) * hs;
    }
  }
  a.g_fine[e] = g;
}

__global__ void k_restrict(int64_t nc, const int64_t* ptr, const int32_t* idx,
                           const double* g_fine, double* g_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double s = 0.0;
  for (int64_t q = ptr[c]; q < ptr[c + 1]; ++q) s += g_fine[idx[q]];
  g_out[c] = s;
}

__global__ void k_d2f(const double* in, float* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

__global__ void k_add_int(int32_t* p, int32_t v) { *p += v; }
__global__ void k_set_int(int32_t* p, int32_t v) { *p = v; }

__global__ void k_copy_f4(const float4* __restrict__ src, float4* __restrict__ dst,
                          int64_t n4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}


int lpr_of(int S_pad) { return S_pad >= kTile ? 32 : S_pad / 4; }

}  // namespace

int launch_step(const StepArgs& a, int S_pad, cudaStream_t st) {
  const int lpr = lpr_of(S_pad);
  const int rows_per_block = kWarps * (32 / lpr);
  dim3 grid((a.K.n + rows_per_block - 1) / rows_per_block, S_pad >= kTile ? S_pad / kTile : 1);
  const int B = a.batch == 4 ? 4 : 8;
  switch (lpr * 16 + B) {
#define MG_CASE(L_, B_) case L_ * 16 + B_: k_step<L_, B_><<<grid, kThreads, 0, st>>>(a); break;
    MG_CASE(32, 4) MG_CASE(32, 8) MG_CASE(16, 4) MG_CASE(16, 8) MG_CASE(8, 4) MG_CASE(8, 8)
    MG_CASE(4, 4) MG_CASE(4, 8) MG_CASE(2, 4) MG_CASE(2, 8) MG_CASE(1, 4) MG_CASE(1, 8)
#undef MG_CASE
    default: return MG_ERR_ARG;
  }
  return check_launch();
}

int launch_step_single(const StepArgs& a, int shot, cudaStream_t st) {
  k_step_single<<<(a.K.n + 255) / 256, 256, 0, st>>>(a, shot);
  return check_launch();
}

int launch_tangent(const TangentArgs& a, int S_pad, cudaStream_t st) {
  const int lpr = lpr_of(S_pad);
  const int rows_per_block = kWarps * (32 / lpr);
  dim3 grid((a.f.K.n + rows_per_block - 1) / rows_per_block, S_pad >= kTile ? S_pad / kTile : 1);
  const int B = a.f.batch == 4 ? 4 : 8;
  switch (lpr * 16 + B) {
#define MG_CASE(L_, B_) case L_ * 16 + B_: k_tangent<L_, B_><<<grid, kThreads, 0, st>>>(a); break;
    MG_CASE(32, 4) MG_CASE(32, 8) MG_CASE(16, 4) MG_CASE(16, 8) MG_CASE(8, 4) MG_CASE(8, 8)
    MG_CASE(4, 4) MG_CASE(4, 8) MG_CASE(2, 4) MG_CASE(2, 8) MG_CASE(1, 4) MG_CASE(1, 8)
#undef MG_CASE
    default: return MG_ERR_ARG;
  }
  return check_launch();
}

int launch_adjoint(const AdjointArgs& a, int S_pad, cudaStream_t st) {
  const int lpr = lpr_of(S_pad);
  const int rows_per_block = kWarps * (32 / lpr);
  dim3 grid((a.K.n + rows_per_block - 1) / rows_per_block, S_pad >= kTile ? S_pad / kTile : 1);
  const int B = a.batch == 4 ? 4 : 8;
  switch (lpr * 16 + B) {
#define MG_CASE(L_, B_) case L_ * 16 + B_: k_adjoint<L_, B_><<<grid, kThreads, 0, st>>>(a); break;
    MG_CASE(32, 4) MG_CASE(32, 8) MG_CASE(16, 4) MG_CASE(16, 8) MG_CASE(8, 4) MG_CASE(8, 8)
    MG_CASE(4, 4) MG_CASE(4, 8) MG_CASE(2, 4) MG_CASE(2, 8) MG_CASE(1, 4) MG_CASE(1, 8)
#undef MG_CASE
    default: return MG_ERR_ARG;
  }
  return check_launch();
}

int launch_coefs(const CoefArgs& a, cudaStream_t st) {
  k_coefs<<<(a.n + 255) / 256, 256, 0, st>>>(a);
  return check_launch();
}

int launch_tangent_coefs(const TangentCoefArgs& a, cudaStream_t st) {
  k_tangent_coefs<<<(a.c.n + 255) / 256, 256, 0, st>>>(a);
  return check_launch();
}

int launch_cfl_reduce(int32_t n, const double* row_abs, const double* mass,
                      double* out, cudaStream_t st) {
  if (cudaMemsetAsync(out, 0, sizeof(double), st) != cudaSuccess) return MG_ERR_CUDA;
  k_cfl_reduce<<<(n + 255) / 256, 256, 0, st>>>(n, row_abs, mass,
                                                 reinterpret_cast<unsigned long long*>(out));
  return check_launch();
}

int launch_cell_gradient(const GradArgs& a, cudaStream_t st) {
  k_cell_gradient<<<(unsigned)((a.m + 255) / 256), 256, 0, st>>>(a);
  return check_launch();
}

int launch_restrict(int64_t nc, const int64_t* ptr, const int32_t* idx,
                    const double* g_fine, double* g_out, cudaStream_t st) {
  k_restrict<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(nc, ptr, idx, g_fine, g_out);
  return check_launch();
}

int launch_d2f(const double* in, float* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return MG_OK;
  k_d2f<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return check_launch();
}

int launch_add_int(int32_t* p, int32_t v, cudaStream_t st) {
  k_add_int<<<1, 1, 0, st>>>(p, v);
  return check_launch();
}

int launch_set_int(int32_t* p, int32_t v, cudaStream_t st) {
  k_set_int<<<1, 1, 0, st>>>(p, v);
  return check_launch();
}

int launch_copy_f4(const float* src, float* dst, int64_t n_floats, cudaStream_t st) {
  const int64_t n4 = n_floats / 4;
  if (n4 <= 0) return MG_OK;
  const int64_t blocks = (n4 + 255) / 256;
  k_copy_f4<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(
      reinterpret_cast<const float4*>(src), reinterpret_cast<float4*>(dst), n4);
  return check_launch();
}

}  // namespace mg
