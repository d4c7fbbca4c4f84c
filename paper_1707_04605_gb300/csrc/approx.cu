// The paper's approximate Jacobian (App. A.1-A.3: auxiliary system,
// Green's functions by reciprocity, multigrid approach, Eq. (approx_2)).
//
// The leapfrog is linear and time invariant with a symmetric system matrix
// A(z), so the impulse response H_{r,i} from node i to receiver r equals
// H_{i,r}.  The trace derivative with respect to coarse cell j is
// approximated (approx_2) by auxiliary sources on the d+1 corner nodes of
// the cell with the lumped coarse mass |T'_j|/(d+1):
//   L'_j = (|T'_j|/(d+1)) sum_{i in corners(j)} phi_i,
//   phi_i = H_{i,r} * z_i,  z_i[l] = -(p_{l+1} - 2 p_l + p_{l-1})_i / dt^2.
// Per shot chunk: one batched forward with the wavelet at the shots'
// sources and one with a unit impulse at their receivers, both recorded at
// every corner node of the level; the convolutions run in the frequency
// domain (cuFFT, FP32, zero-padded to a length >= 2 nt + 2 so that the first
// nt samples of the linear convolution are exact), the second difference as
// the factor -(1 - e^{-i w})^2 / dt^2.  Optional outputs: the node
// responses phi, and the projected approximate Jacobian
// <u_s, L'_j(s)>_k (Sec. II, projected data) accumulated in FP64.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mgwave.h"
#include "mesh_view.h"
#include "mg_internal.h"

namespace mg {
namespace {

// Smallest 2^a 3^b 5^c 7^d >= 2 nt + 2: z carries nt + 2 samples (the second
// difference reaches two steps past the last one), so circular products of
// this length leave the first nt samples of the linear convolution intact.
int nfft_for(int nt) {
  for (int n = 2 * nt + 2;; ++n) {
    int m = n;
    for (int p : {2, 3, 5, 7})
      while (m % p == 0) m /= p;
    if (m == 1) return n;
  }
}

// rows of `dst` (pitch `pitch` floats) <- rows of src ([rows][nt]), zero tail
__global__ void k_pad(int64_t rows, int nt, int pitch, const float* __restrict__ src,
                      float* __restrict__ dst) {
  const int64_t r = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
  if (r >= rows) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < pitch; c += gridDim.x * blockDim.x)
    dst[r * pitch + c] = c < nt ? src[r * nt + c] : 0.0f;
}

// Phi = G * Y * ( -(1 - e^{-i w_k})^2 / dt^2 ) / nfft   (in place in G)
__global__ void k_mul_spectra(int64_t rows, int nc, int nfft, double dt, cufftComplex* G,
                              const cufftComplex* __restrict__ Y) {
  const int64_t total = rows * (int64_t)nc;
  const double two_pi = 6.283185307179586476925286766559;
  const float scale = (float)(1.0 / ((double)nfft * dt * dt));
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % nc);
    double sn, cs;
    sincos(two_pi * k / nfft, &sn, &cs);
    // (1 - e^{-iw})^2 = (1 - cos w + i sin w)^2
    const double ar = 1.0 - cs, ai = sn;
    const float fr = (float)(-(ar * ar - ai * ai)), fi = (float)(-(2.0 * ar * ai));
    const cufftComplex y = Y[q], g = G[q];
    const float zr = y.x * fr - y.y * fi, zi = y.x * fi + y.y * fr;
    G[q] = make_cuComplex((g.x * zr - g.y * zi) * scale, (g.x * zi + g.y * zr) * scale);
  }
}

// P[k][s][i] = <u_s, phi_{s,i}>_k (FP64), one block per (s, i)
__global__ void __launch_bounds__(256) k_project_nodes(int S, int N, int nt, int pitch, double dt,
                                                       const float* __restrict__ u,
                                                       const float* __restrict__ phi,
                                                       double* __restrict__ P, int s0,
                                                       int S_total) {
  __shared__ double a1[256], a2[256];
  const int s = blockIdx.y, i = blockIdx.x;
  const float* us = u + (size_t)(s0 + s) * nt;
  const float* ph = phi + ((size_t)s * N + i) * pitch;
  double x1 = 0.0, x2 = 0.0;
  for (int l = threadIdx.x; l < nt; l += 256) {
    const double ab = (double)us[l] * (double)ph[l];
    x1 += ab;
    x2 += (double)(l + 1) * ab;
  }
  a1[threadIdx.x] = x1;
  a2[threadIdx.x] = x2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      a1[threadIdx.x] += a1[threadIdx.x + w];
      a2[threadIdx.x] += a2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double T = (double)nt * dt;
    P[(size_t)(s0 + s) * N + i] = dt * a1[0];
    P[(size_t)S_total * N + (size_t)(s0 + s) * N + i] = dt * (dt * a2[0]) / T;
  }
}

// Lp[k][s][j] = vol_j / (d+1) sum_{v in corners(j)} P[k][s][node(v)]
__global__ void k_cells(int S, int64_t nl, int k1, const int32_t* __restrict__ corner_node,
                        const double* __restrict__ vol, int N, const double* __restrict__ P,
                        double* __restrict__ Lp) {
  const int64_t total = 2 * (int64_t)S * nl;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = q % nl;
    const int64_t ks = q / nl;  // k * S + s
    double acc = 0.0;
    for (int a = 0; a < k1; ++a) acc += P[ks * N + corner_node[j * k1 + a]];
    Lp[q] = vol[j] / k1 * acc;
  }
}

// dst[s][i][l] = phi rows (pitch) for l < nt
__global__ void k_unpad(int64_t rows, int nt, int pitch, const float* __restrict__ src,
                        float* __restrict__ dst) {
  const int64_t r = blockIdx.y + (int64_t)blockIdx.z * gridDim.y;
  if (r >= rows) return;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nt; c += gridDim.x * blockDim.x)
    dst[r * nt + c] = src[r * pitch + c];
}

dim3 row_grid(int64_t rows, int cols) {
  const unsigned gx = (unsigned)std::min<int64_t>((cols + 255) / 256, 64);
  const unsigned gy = (unsigned)std::min<int64_t>(rows, 65535);
  const unsigned gz = (unsigned)((rows + gy - 1) / gy);
  return dim3(gx, gy, gz);
}

struct Dev {  // stream-ordered device scratch released at scope exit
  cudaStream_t st;
  std::vector<void*> p;
  explicit Dev(cudaStream_t s) : st(s) {}
  ~Dev() {
    for (void* q : p) cudaFreeAsync(q, st);
  }
  template <class T>
  T* get(size_t n) {
    void* q = nullptr;
    if (cudaMallocAsync(&q, std::max<size_t>(n, 1) * sizeof(T), st) != cudaSuccess) return nullptr;
    p.push_back(q);
    return static_cast<T*>(q);
  }
};

struct Plan {
  cufftHandle h = 0;
  bool ok = false;
  ~Plan() {
    if (ok) cufftDestroy(h);
  }
};

}  // namespace
}  // namespace mg

extern "C" int mg_approx_jacobian(mg_mesh* M, int level, const double* eps, const mg_shots* shots,
                                  const double* wavelet, double dt, int nt, const float* u,
                                  double* Lp, float* phi, int32_t* nodes, int64_t* n_nodes,
                                  size_t mem_budget, void* stream, int flags) {
  using namespace mg;
  if (!M || !eps || !shots || !wavelet || nt < 1 || !(dt > 0.0) || !n_nodes) return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL)) return MG_ERR_UNSUPPORTED;
  if (Lp && !u) return MG_ERR_ARG;
  const HostMesh* hm = host_mesh(M);
  if (level < 0 || level >= hm->n_levels) return MG_ERR_ARG;
  const int S = shots->n_shots;
  if (S < 1 || !shots->src || !shots->rec_ptr || !shots->rec) return MG_ERR_ARG;
  for (int s = 0; s < S; ++s)
    if (shots->rec_ptr[s] != s || shots->rec_ptr[s + 1] != s + 1) return MG_ERR_UNSUPPORTED;
  const int k1 = hm->dim + 1;
  const int64_t nl = hm->n_cells_level[level];
  // corners of every level cell: descendant vertices used by one descendant
  std::vector<std::vector<int32_t>> verts(nl);
  std::vector<double> vol(nl, 0.0);
  for (int64_t e = 0; e < hm->m; ++e) {
    const int32_t c = hm->ancestors[level][e];
    vol[c] += hm->cell_vol[e];
    for (int a = 0; a < k1; ++a) verts[c].push_back(hm->cells[(size_t)e * k1 + a]);
  }
  std::vector<int32_t> corner_rows((size_t)nl * k1);
  std::vector<int32_t> all_rows;
  for (int64_t c = 0; c < nl; ++c) {
    auto& v = verts[c];
    std::sort(v.begin(), v.end());
    int found = 0;
    for (size_t i = 0; i < v.size();) {
      size_t j = i;
      while (j < v.size() && v[j] == v[i]) ++j;
      if (j - i == 1) {
        if (found == k1) return MG_ERR_NESTING;
        corner_rows[(size_t)c * k1 + found++] = v[i];
      }
      i = j;
    }
    if (found != k1) return MG_ERR_NESTING;  // not a regular (red) refinement
    std::vector<int32_t>().swap(v);
  }
  all_rows = corner_rows;
  std::sort(all_rows.begin(), all_rows.end());
  all_rows.erase(std::unique(all_rows.begin(), all_rows.end()), all_rows.end());
  const int N = (int)all_rows.size();
  std::vector<int32_t> corner_node(corner_rows.size());
  for (size_t q = 0; q < corner_rows.size(); ++q)
    corner_node[q] = (int32_t)(std::lower_bound(all_rows.begin(), all_rows.end(), corner_rows[q]) -
                               all_rows.begin());
  std::vector<int32_t> node_ids(N);
  for (int i = 0; i < N; ++i) node_ids[i] = hm->iperm[all_rows[i]];
  if (nodes) std::memcpy(nodes, node_ids.data(), N * sizeof(int32_t));
  *n_nodes = N;
  if (!Lp && !phi) return MG_OK;

  int dev_prev = 0;
  if (cudaGetDevice(&dev_prev) != cudaSuccess) return MG_ERR_CUDA;
  if (cudaSetDevice(mesh_device(M)) != cudaSuccess) return MG_ERR_CUDA;
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{dev_prev};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool host = flags & MG_HOST_PTRS;
  const int fl = flags & MG_ALLOW_CFL;
  Dev D(st);
  // inputs on the device
  const double* eps_d = eps;
  const double* wav_d = wavelet;
  const float* u_d = u;
  if (host) {
    double* e = D.get<double>(hm->m);
    double* w = D.get<double>(nt);
    if (!e || !w) return MG_ERR_OOM;
    if (cudaMemcpyAsync(e, eps, hm->m * sizeof(double), cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(w, wavelet, nt * sizeof(double), cudaMemcpyHostToDevice, st))
      return MG_ERR_CUDA;
    eps_d = e;
    wav_d = w;
    if (u) {
      float* uu = D.get<float>((size_t)S * nt);
      if (!uu) return MG_ERR_OOM;
      if (cudaMemcpyAsync(uu, u, (size_t)S * nt * sizeof(float), cudaMemcpyHostToDevice, st))
        return MG_ERR_CUDA;
      u_d = uu;
    }
  }
  std::vector<double> imp_h(nt, 0.0);
  imp_h[0] = 1.0;
  double* imp = D.get<double>(nt);
  int32_t* d_corner = D.get<int32_t>(corner_node.size());
  double* d_vol = D.get<double>(nl);
  double* P = Lp ? D.get<double>(2 * (size_t)S * N) : nullptr;
  if (!imp || !d_corner || !d_vol || (Lp && !P)) return MG_ERR_OOM;
  if (cudaMemcpyAsync(imp, imp_h.data(), nt * sizeof(double), cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_corner, corner_node.data(), corner_node.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_vol, vol.data(), nl * sizeof(double), cudaMemcpyHostToDevice, st))
    return MG_ERR_CUDA;

  const int nfft = nfft_for(nt);
  const int nc = nfft / 2 + 1;
  const int pitch = 2 * nc;  // floats per padded row (in-place R2C)
  // per shot: traces Y, G ([N][nt]) and the padded rows ([N][pitch]) x 2
  const size_t per_shot = (size_t)N * (2 * (size_t)nt + 2 * (size_t)pitch) * sizeof(float);
  const size_t budget = mem_budget ? mem_budget : ((size_t)8 << 30);
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(S, budget / per_shot));
  float* Y = D.get<float>((size_t)chunk * N * nt);
  float* G = D.get<float>((size_t)chunk * N * nt);
  float* Yp = D.get<float>((size_t)chunk * N * pitch);
  float* Gp = D.get<float>((size_t)chunk * N * pitch);
  float* phi_dev = (phi && host) ? D.get<float>((size_t)chunk * N * nt) : nullptr;
  if (!Y || !G || !Yp || !Gp || (phi && host && !phi_dev)) return MG_ERR_OOM;

  std::vector<int32_t> srcA, srcB, rec((size_t)chunk * N);
  std::vector<int64_t> ptr(chunk + 1);
  for (int s0 = 0; s0 < S; s0 += chunk) {
    const int cs = std::min(chunk, S - s0);
    const int64_t rows = (int64_t)cs * N;
    srcA.assign(shots->src + s0, shots->src + s0 + cs);
    srcB.resize(cs);
    for (int s = 0; s < cs; ++s) {
      srcB[s] = shots->rec[s0 + s];
      ptr[s] = (int64_t)s * N;
      for (int i = 0; i < N; ++i) rec[(size_t)s * N + i] = node_ids[i];
    }
    ptr[cs] = rows;
    mg_shots A{cs, srcA.data(), ptr.data(), rec.data()};
    mg_shots B{cs, srcB.data(), ptr.data(), rec.data()};
    int rc = mg_forward(M, eps_d, &A, wav_d, dt, nt, Y, 0, st, fl);
    if (rc) return rc;
    rc = mg_forward(M, eps_d, &B, imp, dt, nt, G, 0, st, fl);
    if (rc) return rc;
    const dim3 gp = row_grid(rows, pitch);
    k_pad<<<gp, 256, 0, st>>>(rows, nt, pitch, Y, Yp);
    k_pad<<<gp, 256, 0, st>>>(rows, nt, pitch, G, Gp);
    if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
    Plan fwd, inv;
    int n[1] = {nfft};
    int inembed[1] = {pitch}, onembed[1] = {nc};
    if (cufftPlanMany(&fwd.h, 1, n, inembed, 1, pitch, onembed, 1, nc, CUFFT_R2C, (int)rows) !=
        CUFFT_SUCCESS)
      return MG_ERR_CUDA;
    fwd.ok = true;
    if (cufftPlanMany(&inv.h, 1, n, onembed, 1, nc, inembed, 1, pitch, CUFFT_C2R, (int)rows) !=
        CUFFT_SUCCESS)
      return MG_ERR_CUDA;
    inv.ok = true;
    cufftSetStream(fwd.h, st);
    cufftSetStream(inv.h, st);
    if (cufftExecR2C(fwd.h, Yp, reinterpret_cast<cufftComplex*>(Yp)) != CUFFT_SUCCESS ||
        cufftExecR2C(fwd.h, Gp, reinterpret_cast<cufftComplex*>(Gp)) != CUFFT_SUCCESS)
      return MG_ERR_CUDA;
    k_mul_spectra<<<152 * 16, 256, 0, st>>>(rows, nc, nfft, dt,
                                             reinterpret_cast<cufftComplex*>(Gp),
                                             reinterpret_cast<const cufftComplex*>(Yp));
    if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
    if (cufftExecC2R(inv.h, reinterpret_cast<cufftComplex*>(Gp), Gp) != CUFFT_SUCCESS)
      return MG_ERR_CUDA;
    add_launches(M, 6);
    if (Lp) {
      k_project_nodes<<<dim3(N, cs), 256, 0, st>>>(cs, N, nt, pitch, dt, u_d, Gp, P, s0, S);
      if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
    }
    if (phi) {
      float* out = host ? phi_dev : phi + (size_t)s0 * N * nt;
      k_unpad<<<row_grid(rows, nt), 256, 0, st>>>(rows, nt, pitch, Gp, out);
      if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
      if (host && cudaMemcpyAsync(phi + (size_t)s0 * N * nt, phi_dev,
                                  (size_t)rows * nt * sizeof(float), cudaMemcpyDeviceToHost, st))
        return MG_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return MG_ERR_CUDA;  // plans are released
  }
  if (Lp) {
    double* out = host ? D.get<double>(2 * (size_t)S * nl) : Lp;
    if (!out) return MG_ERR_OOM;
    k_cells<<<152 * 8, 256, 0, st>>>(S, nl, k1, d_corner, d_vol, N, P, out);
    if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
    if (host && cudaMemcpyAsync(Lp, out, 2 * (size_t)S * nl * sizeof(double),
                                cudaMemcpyDeviceToHost, st))
      return MG_ERR_CUDA;
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}
