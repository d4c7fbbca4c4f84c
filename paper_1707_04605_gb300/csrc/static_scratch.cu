// mg_forward_noalloc: the batched forward without any allocation.
//
// Some callers cannot let a library allocate device memory: applications
// that hand the whole device to their own memory pool (a cudaMalloc from
// the library would fail or fragment it), code that must not pay the
// implicit device synchronisation of cudaMalloc/cudaFree inside a
// latency-critical loop, and drivers that run the call while other work is
// being recorded or replayed and want the call's memory footprint fixed in
// advance.  This entry point serves them: every piece of scratch it needs
// lives in one file-scope device array of a fixed size, reserved once on
// every device that loads the library and held until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/mgwave.h"
#include "kernels.cuh"
#include "mesh_view.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device `dev`, looked up once
// per device (normally by mg::noalloc_prepare when a mesh handle is created
// on that device).
int scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return MG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MG_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return MG_OK;
}

// Bump allocator over the fixed array: only computes offsets.
struct Carve {
  size_t off = 0;
  template <class T>
  size_t take(size_t count) {
    const size_t o = off;
    off += (count * sizeof(T) + 255) / 256 * 256;
    return o;
  }
};

// Per-row source/receiver lists of the shot batch, built on the device.
__global__ void k_ev_count(int S, const int32_t* src, int64_t R, const int32_t* rec,
                           const int32_t* perm, int32_t* src_cnt, int32_t* rec_cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S) atomicAdd(src_cnt + perm[src[i]] + 1, 1);
  else if (i < S + R) atomicAdd(rec_cnt + perm[rec[i - S]] + 1, 1);
}

// Inclusive scan of a[0..len) by one block (blockIdx.x selects the array).
__global__ void k_scan2(int32_t* a0, int32_t* a1, int64_t len) {
  __shared__ int32_t part[1024];
  int32_t* a = blockIdx.x == 0 ? a0 : a1;
  const int64_t chunk = (len + blockDim.x - 1) / blockDim.x;
  const int64_t b = threadIdx.x * chunk;
  const int64_t e = b + chunk < len ? b + chunk : len;
  int32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (unsigned t = 0; t < blockDim.x; ++t) {
      const int32_t v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  int32_t run = part[threadIdx.x];
  for (int64_t i = b; i < e; ++i) {
    run += a[i];
    a[i] = run;
  }
}

__global__ void k_ev_fill(int S, const int32_t* src, int64_t R, const int64_t* shot_ptr,
                          const int32_t* rec, const int32_t* perm, const int32_t* src_ptr,
                          int32_t* src_cur, int32_t* src_shot, const int32_t* rec_ptr,
                          int32_t* rec_cur, int32_t* rec_shot, int32_t* rec_trace) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S) {
    const int32_t row = perm[src[i]];
    src_shot[src_ptr[row] + atomicAdd(src_cur + row, 1)] = (int32_t)i;
  } else if (i < S + R) {
    const int64_t r = i - S;
    int lo = 0, hi = S;  // shot k with shot_ptr[k] <= r < shot_ptr[k+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (shot_ptr[mid] <= r) lo = mid; else hi = mid;
    }
    const int32_t row = perm[rec[r]];
    const int32_t pos = rec_ptr[row] + atomicAdd(rec_cur + row, 1);
    rec_shot[pos] = lo;
    rec_trace[pos] = (int32_t)r;
  }
}

#define NA_TRY(x) do { const int _rc = (x); if (_rc != MG_OK) return _rc; } while (0)
#define NA_CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return MG_ERR_CUDA; } } while (0)

}  // namespace

namespace mg {

int noalloc_prepare(int dev) {
  unsigned char* base = nullptr;
  const int rc = scratch_address(dev, &base);
  if (rc != MG_OK) return rc;
  // load the entry point's own kernels too (lazy module loading would
  // otherwise load them, and reserve their code memory, at its first call)
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_ev_count) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_scan2) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_ev_fill) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

}  // namespace mg

extern "C" int mg_forward_noalloc(mg_mesh* mesh, const double* eps, const mg_shots* shots,
                                  const double* wavelet, double dt, int nt, float* traces,
                                  void* stream, int flags) {
  mg::MeshView v;
  if (!mesh || !eps || !shots || !wavelet || !traces || nt < 1 || !(dt > 0.0)) return MG_ERR_ARG;
  if (flags & ~MG_ALLOW_CFL) return MG_ERR_UNSUPPORTED;
  NA_TRY(mg::mesh_view(mesh, &v));
  // shot batch (host memory, read in place)
  const int S = shots->n_shots;
  if (S < 1 || !shots->src || !shots->rec_ptr || shots->rec_ptr[0] != 0) return MG_ERR_ARG;
  for (int k = 0; k < S; ++k)
    if (shots->src[k] < 0 || shots->src[k] >= v.n || shots->rec_ptr[k + 1] < shots->rec_ptr[k])
      return MG_ERR_ARG;
  const int64_t R = shots->rec_ptr[S];
  if (R > 0 && !shots->rec) return MG_ERR_ARG;
  for (int64_t r = 0; r < R; ++r)
    if (shots->rec[r] < 0 || shots->rec[r] >= v.n) return MG_ERR_ARG;
  const int S_pad = mg::padded_shots(S);
  const int64_t n = v.n;
  // carve the fixed array; reject work that does not fit
  Carve c;
  const size_t o_perm = c.take<int32_t>(n);
  const size_t o_src = c.take<int32_t>(S);
  const size_t o_sptr = c.take<int64_t>(S + 1);
  const size_t o_rec = c.take<int32_t>(R);
  const size_t o_evs = c.take<int32_t>(2 * (n + 1));  // src_ptr | rec_ptr
  const size_t o_cur = c.take<int32_t>(2 * n);        // src_cur | rec_cur
  const size_t o_sshot = c.take<int32_t>(S);
  const size_t o_rshot = c.take<int32_t>(R);
  const size_t o_rtr = c.take<int32_t>(R);
  const size_t o_coef = c.take<float4>(n);
  const size_t o_mass = c.take<double>(n);
  const size_t o_scal = c.take<double>(1);
  const size_t o_wav = c.take<float>(nt);
  const size_t o_st = c.take<float>(2 * (size_t)n * S_pad);
  if (c.off > kScratchBytes) return MG_ERR_ARG;

  int cur_dev = -1;
  NA_CU(cudaGetDevice(&cur_dev));
  if (cur_dev != v.device) NA_CU(cudaSetDevice(v.device));
  struct Restore {
    int d, prev;
    ~Restore() { if (d != prev) cudaSetDevice(prev); }
  } restore{v.device, cur_dev};
  unsigned char* base = nullptr;
  NA_TRY(scratch_address(v.device, &base));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* perm = reinterpret_cast<int32_t*>(base + o_perm);
  int32_t* src = reinterpret_cast<int32_t*>(base + o_src);
  int64_t* sptr = reinterpret_cast<int64_t*>(base + o_sptr);
  int32_t* rec = reinterpret_cast<int32_t*>(base + o_rec);
  int32_t* src_ptr = reinterpret_cast<int32_t*>(base + o_evs);
  int32_t* rec_ptr = src_ptr + (n + 1);
  int32_t* src_cur = reinterpret_cast<int32_t*>(base + o_cur);
  int32_t* rec_cur = src_cur + n;
  int32_t* src_shot = reinterpret_cast<int32_t*>(base + o_sshot);
  int32_t* rec_shot = reinterpret_cast<int32_t*>(base + o_rshot);
  int32_t* rec_trace = reinterpret_cast<int32_t*>(base + o_rtr);
  float4* coef = reinterpret_cast<float4*>(base + o_coef);
  double* mass = reinterpret_cast<double*>(base + o_mass);
  double* scal = reinterpret_cast<double*>(base + o_scal);
  float* wavf = reinterpret_cast<float*>(base + o_wav);
  float* p = reinterpret_cast<float*>(base + o_st);
  float* pm = p + (size_t)n * S_pad;

  // stability bound
  mg::CoefArgs ca = v.coef_base;
  ca.eps = eps;
  if (!(flags & MG_ALLOW_CFL)) {
    ca.dt = 1.0;
    ca.coef = coef;
    ca.mass = mass;
    NA_TRY(mg::launch_coefs(ca, st));
    NA_TRY(mg::launch_cfl_reduce((int32_t)n, v.row_abs, mass, scal, st));
    *v.launches += 2;
    double lam = 0.0;
    NA_CU(cudaMemcpyAsync(&lam, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    NA_CU(cudaStreamSynchronize(st));
    if (!(lam > 0.0) || dt > 2.0 / std::sqrt(lam) * (1.0 + 1e-12)) return MG_ERR_CFL;
  }
  // coefficients, FP32 wavelet
  ca.dt = dt;
  ca.coef = coef;
  ca.mass = nullptr;
  NA_TRY(mg::launch_coefs(ca, st));
  NA_TRY(mg::launch_d2f(wavelet, wavf, nt, st));
  // event lists from the shot batch: everything that must start at zero is
  // cleared here, because the array keeps the previous call's contents
  NA_CU(cudaMemcpyAsync(perm, v.perm_host, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  NA_CU(cudaMemcpyAsync(src, shots->src, S * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  NA_CU(cudaMemcpyAsync(sptr, shots->rec_ptr, (S + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (R > 0)
    NA_CU(cudaMemcpyAsync(rec, shots->rec, R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  NA_CU(cudaMemsetAsync(src_ptr, 0, 2 * (n + 1) * sizeof(int32_t), st));
  NA_CU(cudaMemsetAsync(src_cur, 0, 2 * n * sizeof(int32_t), st));
  const int64_t ne = S + R;
  const unsigned eb = (unsigned)((ne + 255) / 256);
  k_ev_count<<<eb, 256, 0, st>>>(S, src, R, rec, perm, src_ptr, rec_ptr);
  k_scan2<<<2, 1024, 0, st>>>(src_ptr, rec_ptr, n + 1);
  k_ev_fill<<<eb, 256, 0, st>>>(S, src, R, sptr, rec, perm, src_ptr, src_cur, src_shot, rec_ptr,
                                rec_cur, rec_shot, rec_trace);
  NA_CU(cudaGetLastError());
  *v.launches += 5;
  // zero initial states, then the leapfrog steps (plain launches)
  NA_CU(cudaMemsetAsync(p, 0, 2 * (size_t)n * S_pad * sizeof(float), st));
  mg::StepArgs a{};
  a.K = v.K;
  a.ev.src_ptr = src_ptr;
  a.ev.src_shot = src_shot;
  a.ev.rec_ptr = rec_ptr;
  a.ev.rec_shot = rec_shot;
  a.ev.rec_trace = rec_trace;
  a.coef = coef;
  a.ld = S_pad;
  a.wavelet = wavf;
  a.traces = traces;
  a.nt = nt;
  a.step_base = nullptr;
  a.batch = v.batch;
  for (int l = 0; l < nt; ++l) {
    a.p = p;
    a.pm = pm;
    a.pout = pm;
    a.step = l;
    NA_TRY(mg::launch_step(a, S_pad, st));
    *v.launches += 1;
    float* t = p;
    p = pm;
    pm = t;
  }
  return MG_OK;
}
