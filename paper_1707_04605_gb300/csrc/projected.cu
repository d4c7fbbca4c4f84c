// Projected data (Sec. II, "Projected data"): the two time inner products of
// traces and the trace weights that turn a projected-data cotangent into a
// trace cotangent for the adjoint.
//
// A trace holds one sample per leapfrog step, sample l being the field at
// t_l = (l + 1) dt; T = nt dt.  The integrals are the right-endpoint sums
//   <a, b>_1 = sum_l dt a_l b_l,   <a, b>_2 = (1/T) sum_l dt t_l a_l b_l,
// accumulated in FP64 from FP32 samples.  One block per trace; the partial
// sums are combined in a fixed order, so the result depends on nt alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/mgwave.h"

namespace mg {
namespace {

constexpr int kProjThreads = 256;

// One block per trace: thread k sums samples k, k + 256, ... in FP64, then a
// fixed shared-memory tree combines the 256 partial sums.
__global__ void __launch_bounds__(kProjThreads)
    k_project(const float* __restrict__ a, const float* __restrict__ b, int64_t R, int nt,
              double dt, double* __restrict__ y) {
  __shared__ double s1s[kProjThreads], s2s[kProjThreads];
  const int64_t i = blockIdx.x;
  const float* ai = a + i * nt;
  const float* bi = b + i * nt;
  double s1 = 0.0, s2 = 0.0;
  for (int l = threadIdx.x; l < nt; l += kProjThreads) {
    const double ab = (double)__ldg(ai + l) * (double)__ldg(bi + l);
    s1 += ab;
    s2 += (double)(l + 1) * ab;  // t_l / dt
  }
  s1s[threadIdx.x] = s1;
  s2s[threadIdx.x] = s2;
  __syncthreads();
  for (int w = kProjThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1s[threadIdx.x] += s1s[threadIdx.x + w];
      s2s[threadIdx.x] += s2s[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double T = (double)nt * dt;
    y[i] = dt * s1s[0];
    y[R + i] = dt * (dt * s2s[0]) / T;
  }
}

// w_i(t_l) = dt (z1_i + z2_i t_l / T) u_i(t_l), evaluated in FP64, stored FP32;
// blockIdx.y strides over the traces.
__global__ void k_projected_weights(const float* __restrict__ u, const double* __restrict__ z,
                                    int64_t R, int nt, double dt, float* __restrict__ w) {
  const double T = (double)nt * dt;
  for (int64_t i = blockIdx.y; i < R; i += gridDim.y) {
    const double z1 = __ldg(z + i), z2 = __ldg(z + R + i);
    const float* ui = u + i * nt;
    float* wi = w + i * nt;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nt; l += gridDim.x * blockDim.x) {
      const double t = (double)(l + 1) * dt;
      wi[l] = (float)(dt * (z1 + z2 * t / T) * (double)__ldg(ui + l));
    }
  }
}

int launch_project(const float* a, const float* b, int64_t R, int nt, double dt, double* y,
                   cudaStream_t st) {
  k_project<<<(unsigned)R, kProjThreads, 0, st>>>(a, b, R, nt, dt, y);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

int launch_projected_weights(const float* u, const double* z, int64_t R, int nt, double dt,
                             float* w, cudaStream_t st) {
  const int bx = (int)std::min<int64_t>((nt + 255) / 256, 64);
  const unsigned by = (unsigned)std::min<int64_t>(R, 65535);
  k_projected_weights<<<dim3(bx, by), 256, 0, st>>>(u, z, R, nt, dt, w);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

bool args_ok(int64_t R, int nt, double dt) {
  return R >= 0 && nt >= 1 && dt > 0.0 && dt < 1e300 && R < ((int64_t)1 << 31) &&
         R * (int64_t)nt < ((int64_t)1 << 40);
}

// Host-pointer mode: stream-ordered scratch for the inputs and the output,
// copies in, the kernel, copies out, then a synchronisation.
struct Scratch {
  void* p = nullptr;
  cudaStream_t st;
  explicit Scratch(cudaStream_t s) : st(s) {}
  int get(size_t bytes) {
    return cudaMallocAsync(&p, bytes ? bytes : 16, st) == cudaSuccess ? MG_OK : MG_ERR_OOM;
  }
  ~Scratch() {
    if (p) cudaFreeAsync(p, st);
  }
};

}  // namespace
}  // namespace mg

extern "C" {

int mg_project(const float* a, const float* b, int64_t n_traces, int nt, double dt, double* y,
               void* stream, int flags) {
  if (!mg::args_ok(n_traces, nt, dt)) return MG_ERR_ARG;
  if (flags & ~MG_HOST_PTRS) return MG_ERR_UNSUPPORTED;
  if (n_traces == 0) return MG_OK;  // nothing to read or write (pointers may be null)
  if (!a || !b || !y) return MG_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t tb = (size_t)n_traces * nt * sizeof(float);
  const size_t yb = 2 * (size_t)n_traces * sizeof(double);
  if (!(flags & MG_HOST_PTRS)) return mg::launch_project(a, b, n_traces, nt, dt, y, st);
  mg::Scratch s(st);
  int rc = s.get(2 * tb + yb);
  if (rc) return rc;
  float* da = static_cast<float*>(s.p);
  float* db = da + (size_t)n_traces * nt;
  double* dy = reinterpret_cast<double*>(db + (size_t)n_traces * nt);
  if (cudaMemcpyAsync(da, a, tb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(db, b, tb, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MG_ERR_CUDA;
  rc = mg::launch_project(da, db, n_traces, nt, dt, dy, st);
  if (rc) return rc;
  if (cudaMemcpyAsync(y, dy, yb, cudaMemcpyDeviceToHost, st) != cudaSuccess) return MG_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

int mg_projected_weights(const float* u, const double* z, int64_t n_traces, int nt, double dt,
                         float* w, void* stream, int flags) {
  if (!mg::args_ok(n_traces, nt, dt)) return MG_ERR_ARG;
  if (flags & ~MG_HOST_PTRS) return MG_ERR_UNSUPPORTED;
  if (n_traces == 0) return MG_OK;  // nothing to read or write (pointers may be null)
  if (!u || !z || !w) return MG_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t tb = (size_t)n_traces * nt * sizeof(float);
  const size_t zb = 2 * (size_t)n_traces * sizeof(double);
  if (!(flags & MG_HOST_PTRS)) return mg::launch_projected_weights(u, z, n_traces, nt, dt, w, st);
  mg::Scratch s(st);
  int rc = s.get(2 * tb + zb);
  if (rc) return rc;
  float* du = static_cast<float*>(s.p);
  float* dw = du + (size_t)n_traces * nt;
  double* dz = reinterpret_cast<double*>(dw + (size_t)n_traces * nt);
  if (cudaMemcpyAsync(du, u, tb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dz, z, zb, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MG_ERR_CUDA;
  rc = mg::launch_projected_weights(du, dz, n_traces, nt, dt, dw, st);
  if (rc) return rc;
  if (cudaMemcpyAsync(w, dw, tb, cudaMemcpyDeviceToHost, st) != cudaSuccess) return MG_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

}  // extern "C"
