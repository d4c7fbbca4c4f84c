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
  float out = leap1(c.x, c.y, c.z, self, old, acc);
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

// Lumped conductivity mass R_rr = sum_{e contains r} sigma_e |e|/(d+1): the
// sigma du/dt term of Eq. (pde1), centred in time with the boundary damping.
__device__ __forceinline__ double sigma_mass(const CoefArgs& a, int r) {
  double R = 0.0;
  if (a.sigma)
    for (int64_t q = a.nc_ptr[r]; q < a.nc_ptr[r + 1]; ++q) R += a.sigma[a.nc_cell[q]] * a.nc_w[q];
  return R;
}

__global__ void k_coefs(CoefArgs a) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n) return;
  double m = 0.0, D = 0.0;
  for (int64_t q = a.nc_ptr[r]; q < a.nc_ptr[r + 1]; ++q) m += a.eps[a.nc_cell[q]] * a.nc_w[q];
  if (a.bc == MG_BC_ABC1)
    for (int64_t q = a.nf_ptr[r]; q < a.nf_ptr[r + 1]; ++q)
      D += sqrt(a.eps[a.nf_cell[q]]) * a.nf_w[q];
  D += sigma_mass(a, r);
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
  D += sigma_mass(a.c, r);  // sigma is not a parameter: no dD term
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


}  // namespace

namespace {
__global__ void k_prolong(int64_t m, const int32_t* anc, const double* v, const double* base,
                          double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) out[e] = (base ? base[e] : 0.0) + v[anc[e]];
}
}  // namespace

int launch_prolong(int64_t m, const int32_t* anc, const double* v, const double* base,
                   double* out, cudaStream_t st) {
  k_prolong<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, anc, v, base, out);
  return check_launch();
}

int launch_step_single(const StepArgs& a, int shot, cudaStream_t st) {
  k_step_single<<<(a.K.n + 255) / 256, 256, 0, st>>>(a, shot);
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
