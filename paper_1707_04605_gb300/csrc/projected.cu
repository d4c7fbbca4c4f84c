// Projected data (Sec. II, "Projected data"): the two time inner products of
// traces and the trace weights that turn a projected-data cotangent into a
// trace cotangent for the adjoint.
//
// A trace holds one sample per leapfrog step, sample l being the field at
// t_l = (l + 1) dt; T = nt dt.  The integrals are the right-endpoint sums
//   <a, b>_1 = sum_l dt a_l b_l,   <a, b>_2 = (1/T) sum_l dt t_l a_l b_l,
// accumulated in FP64 from FP32 samples.  One warp per trace: lane k sums
// samples k, k + 32, ...; the 32 partial sums are combined by a fixed
// butterfly, so the result does not depend on the launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mgwave.h"

namespace mg {
namespace {

constexpr int kProjWarps = 8;

__global__ void __launch_bounds__(32 * kProjWarps)
    k_project(const float* __restrict__ a, const float* __restrict__ b, int64_t R, int nt,
              double dt, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kProjWarps + (threadIdx.x >> 5);
  if (i >= R) return;  // whole warps leave together (R is per warp)
  const float* ai = a + i * nt;
  const float* bi = b + i * nt;
  double s1 = 0.0, s2 = 0.0;
  for (int l = lane; l < nt; l += 32) {
    const double ab = (double)__ldg(ai + l) * (double)__ldg(bi + l);
    s1 += ab;
    s2 += (double)(l + 1) * ab;  // t_l / dt
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  }
  if (lane == 0) {
    const double T = (double)nt * dt;
    y[i] = dt * s1;
    y[R + i] = dt * (dt * s2) / T;
  }
}

// w_i(t_l) = dt (z1_i + z2_i t_l / T) u_i(t_l), evaluated in FP64, stored FP32.
__global__ void k_projected_weights(const float* __restrict__ u, const double* __restrict__ z,
                                    int64_t R, int nt, double dt, float* __restrict__ w) {
  const int64_t total = R * (int64_t)nt;
  const double T = (double)nt * dt;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / nt;
    const int l = (int)(q - i * nt);
    const double t = (double)(l + 1) * dt;
    w[q] = (float)(dt * (__ldg(z + i) + __ldg(z + R + i) * t / T) * (double)__ldg(u + q));
  }
}

int launch_project(const float* a, const float* b, int64_t R, int nt, double dt, double* y,
                   cudaStream_t st) {
  const int64_t blocks = (R + kProjWarps - 1) / kProjWarps;
  k_project<<<(unsigned)blocks, 32 * kProjWarps, 0, st>>>(a, b, R, nt, dt, y);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

int launch_projected_weights(const float* u, const double* z, int64_t R, int nt, double dt,
                             float* w, cudaStream_t st) {
  const int64_t total = R * (int64_t)nt;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_projected_weights<<<(unsigned)blocks, 256, 0, st>>>(u, z, R, nt, dt, w);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

bool args_ok(int64_t R, int nt, double dt) {
  return R >= 0 && nt >= 1 && dt > 0.0 && dt < 1e300 && R < ((int64_t)1 << 31) / 32 &&
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
