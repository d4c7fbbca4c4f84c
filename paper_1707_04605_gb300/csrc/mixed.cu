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
                         const float4* __restrict__ p, float4* __restrict__ q, float dt) {
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

// p <- p + dt/C (f delta_src - (R+S) p - sum_{e ni i} sum_k w[e,i,k] q^(k)_e);
// sources and traces of the row's shots
template <int D>
__global__ void k_flux_p(int64_t n, int64_t m, int ld4, const int64_t* __restrict__ nc_ptr,
                         const int32_t* __restrict__ nc_cell, const float* __restrict__ w,
                         const float2* __restrict__ coef, const float4* __restrict__ q,
                         float4* __restrict__ p, const int32_t* __restrict__ src_ptr,
                         const int32_t* __restrict__ src_shot, const int32_t* __restrict__ rec_ptr,
                         const int32_t* __restrict__ rec_shot,
                         const int32_t* __restrict__ rec_trace, float f, float* __restrict__ traces,
                         int nt, int l) {
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
    p[t] = pv;
    const int r0 = __ldg(rec_ptr + i), r1 = __ldg(rec_ptr + i + 1);
    for (int r = r0; r < r1; ++r) {
      const int d = __ldg(rec_shot + r) - 4 * c4;
      if (d < 0 || d > 3) continue;
      const float v = d == 0 ? pv.x : d == 1 ? pv.y : d == 2 ? pv.z : pv.w;
      traces[(int64_t)__ldg(rec_trace + r) * nt + l] = v;
    }
  }
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
  T* get(size_t count) {
    void* x = nullptr;
    if (cudaMallocAsync(&x, std::max<size_t>(count, 1) * sizeof(T), st) != cudaSuccess)
      return nullptr;
    p.push_back(x);
    return static_cast<T*>(x);
  }
};

int grid_for(int64_t total) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
}

}  // namespace
}  // namespace mg

extern "C" int mg_forward_pml(mg_mesh* M, const double* eps, const mg_shots* shots,
                              const double* wavelet, double dt, int nt, const double* xi,
                              const double* zeta, float* traces, void* stream, int flags) {
  using namespace mg;
  if (!M || !eps || !shots || !wavelet || !traces || nt < 1 || !(dt > 0.0)) return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL)) return MG_ERR_UNSUPPORTED;
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
  int dev_prev = 0;
  if (cudaGetDevice(&dev_prev) != cudaSuccess) return MG_ERR_CUDA;
  if (cudaSetDevice(mesh_device(M)) != cudaSuccess) return MG_ERR_CUDA;
  struct Restore {
    int dv;
    ~Restore() { cudaSetDevice(dv); }
  } restore{dev_prev};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool host = flags & MG_HOST_PTRS;
  Scratch X(st);

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
  std::vector<double> zeta_h, xi_h;
  if (zeta) {
    zeta_h.resize((size_t)m * d);
    if (host) std::copy(zeta, zeta + (size_t)m * d, zeta_h.begin());
    else if (cudaMemcpy(zeta_h.data(), zeta, zeta_h.size() * sizeof(double),
                        cudaMemcpyDeviceToHost) != cudaSuccess)
      return MG_ERR_CUDA;
    for (size_t q = 0; q < zeta_h.size(); ++q) {
      if (!(zeta_h[q] >= 0.0) || !std::isfinite(zeta_h[q])) return MG_ERR_ARG;
      damp[q] = (float)zeta_h[q];
    }
  }
  const int ld = S <= 4 ? 4 : ((S + 3) / 4) * 4;
  const int ld4 = ld / 4;
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
  std::vector<float> fl(nt);
  double acc = 0.0;
  for (int l = 0; l < nt; ++l) {
    acc += dt * wav_h[l];
    fl[l] = (float)acc;
  }

  MeshView V;
  if (mesh_view(M, &V) != MG_OK) return MG_ERR_ARG;
  const double* eps_d = eps;
  const double* xi_d = xi;
  if (host) {
    eps_d = X.put(std::vector<double>(eps, eps + m));
    if (xi) xi_d = X.put(std::vector<double>(xi, xi + m));
    if (!eps_d || (xi && !xi_d)) return MG_ERR_OOM;
  }
  if (!(flags & MG_ALLOW_CFL)) {
    double dtc = 0.0;
    const int rc = mg_cfl_dt(M, eps_d, 0, stream, &dtc);
    if (rc) return rc;
    if (dt > dtc * (1.0 + 1e-12)) return MG_ERR_CFL;
  }
  int32_t* d_cells = X.put(hm->cells);
  float* d_grad = X.put(grad);
  float* d_w = X.put(wnc);
  float* d_damp = X.put(damp);
  int32_t *d_sp = X.put(sp), *d_ss = X.put(ss), *d_rp = X.put(rp), *d_rs = X.put(rs),
          *d_rt = X.put(rt);
  float2* coef = X.get<float2>(n);
  float* p = X.get<float>((size_t)n * ld);
  float* q = X.get<float>((size_t)d * m * ld);
  float* tr = host ? X.get<float>((size_t)R * nt) : traces;
  if (!d_cells || !d_grad || !d_w || !d_damp || !d_sp || !d_ss || !d_rp || !d_rs || !d_rt ||
      !coef || !p || !q || !tr)
    return MG_ERR_OOM;
  if (cudaMemsetAsync(p, 0, (size_t)n * ld * sizeof(float), st) ||
      cudaMemsetAsync(q, 0, (size_t)d * m * ld * sizeof(float), st))
    return MG_ERR_CUDA;
  CoefArgs c = V.coef_base;
  c.eps = eps_d;
  k_flux_coefs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, xi_d, dt, coef);
  if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
  const int gq = grid_for(m * ld4), gp = grid_for(n * ld4);
  const float fdt = (float)dt;
  for (int l = 0; l < nt; ++l) {
    if (d == 2) {
      k_flux_q<2><<<gq, 256, 0, st>>>(m, ld4, d_cells, d_grad, d_damp,
                                       reinterpret_cast<const float4*>(p),
                                       reinterpret_cast<float4*>(q), fdt);
      k_flux_p<2><<<gp, 256, 0, st>>>(n, m, ld4, V.coef_base.nc_ptr, V.coef_base.nc_cell, d_w,
                                       coef, reinterpret_cast<const float4*>(q),
                                       reinterpret_cast<float4*>(p), d_sp, d_ss, d_rp, d_rs,
                                       d_rt, fl[l], tr, nt, l);
    } else {
      k_flux_q<3><<<gq, 256, 0, st>>>(m, ld4, d_cells, d_grad, d_damp,
                                       reinterpret_cast<const float4*>(p),
                                       reinterpret_cast<float4*>(q), fdt);
      k_flux_p<3><<<gp, 256, 0, st>>>(n, m, ld4, V.coef_base.nc_ptr, V.coef_base.nc_cell, d_w,
                                       coef, reinterpret_cast<const float4*>(q),
                                       reinterpret_cast<float4*>(p), d_sp, d_ss, d_rp, d_rs,
                                       d_rt, fl[l], tr, nt, l);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
  add_launches(M, 1 + 2 * (int64_t)nt);
  if (host && cudaMemcpyAsync(traces, tr, (size_t)R * nt * sizeof(float), cudaMemcpyDeviceToHost,
                              st) != cudaSuccess)
    return MG_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}
