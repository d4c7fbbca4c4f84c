// Launchers of the row kernels (rows_common.cuh) with plain neighbour
// gathers; a launch that asks for the gather ring (a.ring / a.f.ring > 0)
// goes to kernels_ring.cu.  Also the multi-step cooperative forward.
#include <algorithm>

#include "rows_common.cuh"

namespace mg {
namespace {

// Grid-wide barrier of a cooperative launch: thread 0 of every CTA adds one
// to *count (after a fence that publishes the CTA's stores) and polls it with
// acquire loads until it reaches `target`.  Bounded: past `budget` SM clock
// cycles, or when *status shows that another CTA gave up, the CTA sets
// *status = 1 and every thread of it gets false.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, int* status,
                                             long long budget) {
  __syncthreads();
  int fail = 0;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    const long long t0 = clock64();
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) break;
      if (*reinterpret_cast<volatile int*>(status) != 0) { fail = 1; break; }
      if (clock64() - t0 > budget) {
        atomicExch(status, 1);
        fail = 1;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  return __syncthreads_or(fail) == 0;
}

// pa.steps forward steps from a.step: states x (p_l) and y (p_{l-1}, then
// p_{l+1}) swap roles after every step, as in the stream of single-step
// launches, and every step is the same block computation (same bits).
template <int LPR, int NV>
__global__ void __launch_bounds__(kThreads) k_step_persist(StepArgs a, PersistArgs pa) {
  constexpr int RPB = kWarps * 32 / LPR;
  const int nblk = (a.K.n + RPB - 1) / RPB;
  const unsigned nctas = gridDim.x * gridDim.y;
  const float* x = a.p;
  float* y = a.pout;
  StepArgs b = a;
  for (int j = 0; j < pa.steps; ++j) {
    b.p = x;
    b.pm = y;
    b.pout = y;
    b.step = a.step + j;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) step_rows_block<LPR, NV, 0>(b, blk);
    if (j + 1 < pa.steps &&
        !grid_barrier(pa.count, (unsigned)(j + 1) * (nctas + (unsigned)pa.extra), pa.status,
                      pa.budget))
      return;
    float* t = const_cast<float*>(x);
    x = y;
    y = t;
  }
}

template <int LPR, int NV>
__global__ void __launch_bounds__(kThreads) k_tangent_persist(TangentArgs a, PersistArgs pa) {
  constexpr int RPB = kWarps * 32 / LPR;
  const int nblk = (a.f.K.n + RPB - 1) / RPB;
  const unsigned nctas = gridDim.x * gridDim.y;
  const float* x = a.q;
  float* y = a.qm;
  TangentArgs b = a;
  for (int j = 0; j < pa.steps; ++j) {
    const int l = a.f.step + j;
    b.f.p = pa.seg + (size_t)(l + 1) * pa.state;
    b.f.pm = pa.seg + (size_t)l * pa.state;
    b.f.pout = pa.seg + (size_t)(l + 2) * pa.state;
    b.f.step = l;
    b.q = x;
    b.qm = y;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) tangent_rows_block<LPR, NV, 0>(b, blk);
    if (j + 1 < pa.steps &&
        !grid_barrier(pa.count, (unsigned)(j + 1) * (nctas + (unsigned)pa.extra), pa.status,
                      pa.budget))
      return;
    float* t = const_cast<float*>(x);
    x = y;
    y = t;
  }
}

template <int LPR, int NV>
__global__ void __launch_bounds__(kThreads) k_adjoint_persist(AdjointArgs a, PersistArgs pa) {
  constexpr int RPB = kWarps * 32 / LPR;
  const int nblk = (a.K.n + RPB - 1) / RPB;
  const unsigned nctas = gridDim.x * gridDim.y;
  const float* x = a.mu;
  float* y = a.mu1;
  AdjointArgs b = a;
  for (int j = 0; j < pa.steps; ++j) {
    const int k = a.k - j;
    b.mu = x;
    b.mu1 = y;
    b.pk = pa.seg + (size_t)(k + 1) * pa.state;
    b.k = k;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) adjoint_rows_block<LPR, NV, 0>(b, blk);
    if (j + 1 < pa.steps &&
        !grid_barrier(pa.count, (unsigned)(j + 1) * (nctas + (unsigned)pa.extra), pa.status,
                      pa.budget))
      return;
    float* t = const_cast<float*>(x);
    x = y;
    y = t;
  }
}

// Cooperative launch of a persistent kernel: at most the kernel's occupancy
// times the SM count CTAs (every CTA resident), the barrier counter zeroed
// on the stream first.
template <class A>
int launch_coop(void (*kern)(A, PersistArgs), Shape sh, const A& a, const PersistArgs& pa,
                cudaStream_t st) {
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  const long resident = (long)occ * nsm;
  if (resident < (long)sh.grid.y) return MG_ERR_UNSUPPORTED;
  sh.grid.x = (unsigned)std::min<long>(sh.grid.x, resident / sh.grid.y);
  if (cudaMemsetAsync(pa.count, 0, sizeof(unsigned), st) != cudaSuccess) return MG_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = sh.grid;
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kern, a, pa) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  return check_launch();
}

bool persist_ok(const PersistArgs& pa) {
  return pa.steps >= 1 && pa.count && pa.status && pa.budget >= 1 && pa.extra >= 0;
}

}  // namespace

int rows_tiles(int cols, int nv) { return (int)shape_of(1, cols, nv).grid.y; }

#define MG_PERSIST_SWITCH(KERN, ARGS)                                                    \
  switch (sh.lpr * 8 + sh.nv) {                                                        \
    case 32 * 8 + 1: return launch_coop(KERN<32, 1>, sh, ARGS, pa, st);                \
    case 32 * 8 + 2: return launch_coop(KERN<32, 2>, sh, ARGS, pa, st);                \
    case 32 * 8 + 4: return launch_coop(KERN<32, 4>, sh, ARGS, pa, st);                \
    case 16 * 8 + 1: return launch_coop(KERN<16, 1>, sh, ARGS, pa, st);                \
    case 16 * 8 + 2: return launch_coop(KERN<16, 2>, sh, ARGS, pa, st);                \
    case 16 * 8 + 4: return launch_coop(KERN<16, 4>, sh, ARGS, pa, st);                \
    case 8 * 8 + 1: return launch_coop(KERN<8, 1>, sh, ARGS, pa, st);                  \
    case 8 * 8 + 2: return launch_coop(KERN<8, 2>, sh, ARGS, pa, st);                  \
    case 8 * 8 + 4: return launch_coop(KERN<8, 4>, sh, ARGS, pa, st);                  \
    case 4 * 8 + 1: return launch_coop(KERN<4, 1>, sh, ARGS, pa, st);                  \
    case 4 * 8 + 2: return launch_coop(KERN<4, 2>, sh, ARGS, pa, st);                  \
    case 4 * 8 + 4: return launch_coop(KERN<4, 4>, sh, ARGS, pa, st);                  \
    case 2 * 8 + 1: return launch_coop(KERN<2, 1>, sh, ARGS, pa, st);                  \
    case 2 * 8 + 2: return launch_coop(KERN<2, 2>, sh, ARGS, pa, st);                  \
    case 2 * 8 + 4: return launch_coop(KERN<2, 4>, sh, ARGS, pa, st);                  \
    case 1 * 8 + 1: return launch_coop(KERN<1, 1>, sh, ARGS, pa, st);                  \
    case 1 * 8 + 2: return launch_coop(KERN<1, 2>, sh, ARGS, pa, st);                  \
    case 1 * 8 + 4: return launch_coop(KERN<1, 4>, sh, ARGS, pa, st);                  \
    default: return MG_ERR_ARG;                                                        \
  }

int launch_tangent_persist(const TangentArgs& a, int S_pad, const PersistArgs& pa,
                           cudaStream_t st) {
  const int cols = a.f.cols ? a.f.cols : S_pad;
  const Shape sh = shape_of(a.f.K.n, cols, a.f.batch);
  if (!range_ok(sh, a.f.col0, cols, a.f.ld) || !persist_ok(pa) || !pa.seg || pa.state < 1 ||
      a.f.step < 0)
    return MG_ERR_ARG;
  MG_PERSIST_SWITCH(k_tangent_persist, a)
}

int launch_adjoint_persist(const AdjointArgs& a, int S_pad, const PersistArgs& pa,
                           cudaStream_t st) {
  const int cols = a.cols ? a.cols : S_pad;
  const Shape sh = shape_of(a.K.n, cols, a.batch);
  if (!range_ok(sh, a.col0, cols, a.ld) || !persist_ok(pa) || !pa.seg || pa.state < 1 ||
      a.k - pa.steps < 0)
    return MG_ERR_ARG;
  MG_PERSIST_SWITCH(k_adjoint_persist, a)
}
#undef MG_PERSIST_SWITCH

int launch_step_persist(const StepArgs& a, int S_pad, const PersistArgs& pa, cudaStream_t st) {
  const int cols = a.cols ? a.cols : S_pad;
  Shape sh = shape_of(a.K.n, cols, a.batch);
  if (!range_ok(sh, a.col0, cols, a.ld) || pa.steps < 1 || a.pout != a.pm || !pa.count ||
      !pa.status || pa.budget < 1 || pa.extra < 0)
    return MG_ERR_ARG;
  void (*kern)(StepArgs, PersistArgs) = nullptr;
  switch (sh.lpr * 8 + sh.nv) {
#define MG_P(L, V) case L * 8 + V: kern = k_step_persist<L, V>; break;
    MG_P(32, 1) MG_P(32, 2) MG_P(32, 4) MG_P(16, 1) MG_P(16, 2) MG_P(16, 4)
    MG_P(8, 1) MG_P(8, 2) MG_P(8, 4) MG_P(4, 1) MG_P(4, 2) MG_P(4, 4)
    MG_P(2, 1) MG_P(2, 2) MG_P(2, 4) MG_P(1, 1) MG_P(1, 2) MG_P(1, 4)
#undef MG_P
    default: return MG_ERR_ARG;
  }
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  const long resident = (long)occ * nsm;   // every CTA of a cooperative launch is resident
  if (resident < (long)sh.grid.y) return MG_ERR_UNSUPPORTED;
  sh.grid.x = (unsigned)std::min<long>(sh.grid.x, resident / sh.grid.y);
  if (cudaMemsetAsync(pa.count, 0, sizeof(unsigned), st) != cudaSuccess) return MG_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = sh.grid;
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kern, a, pa) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  return check_launch();
}

int launch_step(const StepArgs& a, int S_pad, cudaStream_t st) {
  if (a.ring) return launch_step_ring(a, S_pad, st);
  const int cols = a.cols ? a.cols : S_pad;
  Shape sh = shape_of(a.K.n, cols, a.batch);
  if (a.sweep > 1) sh.grid.x = (sh.grid.x + a.sweep - 1) / a.sweep;
  if (!range_ok(sh, a.col0, cols, a.ld)) return MG_ERR_ARG;
  cudaError_t err = cudaSuccess;
  // wide lanes: 32-byte accesses need 32-byte aligned rows and columns
  const uintptr_t al = reinterpret_cast<uintptr_t>(a.p) | reinterpret_cast<uintptr_t>(a.pm) |
                       reinterpret_cast<uintptr_t>(a.pout);
  if (a.wide && a.min_blocks == 5 && sh.nv == 2 && !a.hint && !a.stream && a.ld % 8 == 0 &&
      a.col0 % 8 == 0 && al % 32 == 0) {
    switch (sh.lpr) {
      case 32: err = launch_ex(k_step_rows_w<32, 5>, sh.grid, a.pdl, 0, st, a); break;
      case 16: err = launch_ex(k_step_rows_w<16, 5>, sh.grid, a.pdl, 0, st, a); break;
      case 8: err = launch_ex(k_step_rows_w<8, 5>, sh.grid, a.pdl, 0, st, a); break;
      case 4: err = launch_ex(k_step_rows_w<4, 5>, sh.grid, a.pdl, 0, st, a); break;
      case 2: err = launch_ex(k_step_rows_w<2, 5>, sh.grid, a.pdl, 0, st, a); break;
      case 1: err = launch_ex(k_step_rows_w<1, 5>, sh.grid, a.pdl, 0, st, a); break;
      default: return MG_ERR_ARG;
    }
  } else if (a.min_blocks == 5) {
    MG_ROWS_SWITCH_M(k_step_rows, 5, 0, 1, a.pdl, a)
  } else if (a.min_blocks == 0) {
    MG_ROWS_SWITCH_M(k_step_rows, 1, 0, 1, a.pdl, a)
  } else {
    return MG_ERR_ARG;
  }
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

int launch_tangent(const TangentArgs& a, int S_pad, cudaStream_t st) {
  if (a.f.ring) return launch_tangent_ring(a, S_pad, st);
  const int cols = a.f.cols ? a.f.cols : S_pad;
  const Shape sh = shape_of(a.f.K.n, cols, a.f.batch);
  if (!range_ok(sh, a.f.col0, cols, a.f.ld)) return MG_ERR_ARG;
  cudaError_t err = cudaSuccess;
  if (a.f.min_blocks == 5) {
    MG_ROWS_SWITCH_M(k_tangent_rows, 5, 0, 2, a.f.pdl, a)
  } else if (a.f.min_blocks == 0) {
    MG_ROWS_SWITCH_M(k_tangent_rows, 1, 0, 2, a.f.pdl, a)
  } else {
    return MG_ERR_ARG;
  }
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

int launch_tangent_kept(const TangentArgs& a, int S_pad, cudaStream_t st) {
  if (a.f.ring) return launch_tangent_kept_ring(a, S_pad, st);
  const int cols = a.f.cols ? a.f.cols : S_pad;
  const Shape sh = shape_of(a.f.K.n, cols, a.f.batch);
  if (!range_ok(sh, a.f.col0, cols, a.f.ld) || !a.pk1) return MG_ERR_ARG;
  cudaError_t err = cudaSuccess;
  MG_ROWS_SWITCH(k_tangent_kept_rows, 0, 1, a.f.pdl, a)
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

int launch_adjoint(const AdjointArgs& a, int S_pad, cudaStream_t st) {
  if (a.ring) return launch_adjoint_ring(a, S_pad, st);
  const int cols = a.cols ? a.cols : S_pad;
  const Shape sh = shape_of(a.K.n, cols, a.batch);
  if (!range_ok(sh, a.col0, cols, a.ld)) return MG_ERR_ARG;
  cudaError_t err = cudaSuccess;
  if (a.min_blocks == 6) {
    MG_ROWS_SWITCH_M(k_adjoint_rows, 6, 0, 1, a.pdl, a)
  } else if (a.min_blocks == 5) {
    MG_ROWS_SWITCH_M(k_adjoint_rows, 5, 0, 1, a.pdl, a)
  } else if (a.min_blocks == 0) {
    MG_ROWS_SWITCH_M(k_adjoint_rows, 1, 0, 1, a.pdl, a)
  } else {
    return MG_ERR_ARG;
  }
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

}  // namespace mg
