// Forward leapfrog step on row tiles staged in shared memory by the bulk
// copy engine (TMA), with a producer warp and consumer warps per CTA.
//
// The step p_{l+1} = alpha p_l - beta p_{l-1} - gamma (K p_l - s_l e_src)
// (App. A, Eqs. (leap-frog1)-(leap-frog2) with the flux eliminated) reads
// every row of p_l once per stiffness entry that references it.  The row
// kernels fetch those gathers through L1/L2 one neighbour at a time per
// lane; here a CTA owns a contiguous range of row tiles (HostTiles: P rows
// and the halo rows their stencils reach, 16-bit local indices) and sweeps
// them as work items of 32 shot columns:
//
//  * the producer warp copies, per item, the tile's local stiffness
//    (indices and values) and the 32-column segments of its own and halo
//    rows of p_l into one of two shared-memory buffers with
//    cp.async.bulk, all completing on the buffer's `full` mbarrier;
//  * the consumer warps wait on `full`, compute the tile's rows for those
//    columns from shared memory (8 lanes per row, one float4 of shots per
//    lane, entries read by all 8 lanes of a row at once), read p_{l-1},
//    the coefficients and the source/receiver lists from global memory,
//    store p_{l+1} and the traces, and release the buffer on its `empty`
//    mbarrier while the producer already fills the other one.
//
// Measured on GB300 it is far slower than the row kernels (ellipsoid_3d
// forward 2620 us per step with 128-row tiles against 538 us; ncu: issue
// 12%, DRAM 9% of peak, the copy engine taking one 128-byte row copy per
// ~70 SM cycles): per-row bulk copies are too small for the copy engine.
// It is kept as a tested, bit-identical variant (mg_mesh_set_tma_tiles),
// not as an autotuner candidate.
//
// Each p_l row is brought on chip once per tile that references it (the
// halo ratio of the tiling, about 3 for 128-row tiles of the 3D mesh)
// instead of once per stiffness entry, and all of a tile's copies are in
// flight together without holding registers.  The arithmetic per row is
// the row kernels' (diagonal first, the entries in slice order, the same
// FMAs), so the traces carry the same bits.  Every mbarrier wait is bounded:
// on time-out the thread records 1 in the status word and leaves, and the
// producer waits (bounded) for its copies in flight before it leaves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/mgwave.h"
#include "async_copy.cuh"
#include "device_util.cuh"
#include "kernels.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

using namespace dev;
using namespace ac;

constexpr int kCW = 8;                  // consumer warps
constexpr int kTmaThreads = 32 * (kCW + 1);
constexpr int kHW = 32;                 // shot columns per work item
constexpr int kLPR = kHW / 4;           // lanes per row (one float4 each)
constexpr int kRPW = 32 / kLPR;         // rows per consumer warp and pass
constexpr int kRPP = kCW * kRPW;        // rows per pass of the consumers
constexpr int kBatch = 8;               // producer: row copies per lane per batch

__host__ __device__ __forceinline__ size_t al128(size_t x) { return (x + 127) / 128 * 128; }

// Shared memory: two buffers of [rows of the tile and its halo][kHW]
// floats of p_l, then the tile's local indices and values; then 4
// mbarriers.
struct TmaLayout {
  size_t idx, val, buf, bars, total;
};

__host__ __device__ __forceinline__ TmaLayout tma_layout(const DevTiles& T) {
  TmaLayout L;
  L.idx = al128((size_t)(T.P + T.max_halo) * kHW * sizeof(float));
  L.val = L.idx + al128((size_t)T.max_ell * sizeof(uint16_t));
  L.buf = L.val + al128((size_t)T.max_ell * sizeof(float));
  L.bars = 2 * L.buf;
  L.total = L.bars + 4 * sizeof(uint64_t);
  return L;
}

__device__ __forceinline__ void grid_dep_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Shot s of the item as component d of this lane's float4, or false.
__device__ __forceinline__ bool mine(int s, int col0, int lr, int& d) {
  const int rel = s - col0;
  if (rel < 0 || rel >= kHW || rel / 4 != lr) return false;
  d = rel % 4;
  return true;
}

__global__ void __launch_bounds__(kTmaThreads, 1) k_step_tma(StepArgs a, DevTiles T, int* err,
                                                             int tiles_per_cta) {
  extern __shared__ __align__(128) unsigned char sm[];
  const TmaLayout L = tma_layout(T);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* empty = full + 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cols = a.cols ? a.cols : a.ld;
  const int nchunk = cols / kHW;
  const int t_begin = blockIdx.x * tiles_per_cta;
  const int t_end = min(t_begin + tiles_per_cta, T.n_tiles);
  if (t_begin >= t_end) return;                     // the whole CTA leaves
  const int n_items = (t_end - t_begin) * nchunk;
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], kCW);
    mbar_init(&empty[1], kCW);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dep_sync();                                  // p_l written, p_{l-1} free to overwrite
  const int64_t n = a.K.n;

  if (warp == kCW) {
    // ------------------------------------------------------------ producer
    int issued = 0;
    for (int i = 0; i < n_items; ++i) {
      const int b = i & 1;
      const uint32_t round = (uint32_t)(i >> 1);
      if (i >= 2) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&empty[b], (round - 1) & 1));
        if (!ok) {
          if (lane == 0) atomicExch(err, 1);
          break;
        }
      }
      const int t = t_begin + i / nchunk, ch = i % nchunk;
      const int64_t t0 = (int64_t)t * T.P;
      const int Pt = (int)(n - t0 < (int64_t)T.P ? n - t0 : (int64_t)T.P);
      const int nh = __ldg(T.halo_cnt + t);
      const int64_t e0 = __ldg(T.ell_off + t);
      const int ne = (int)(__ldg(T.ell_off + t + 1) - e0);
      const int64_t h0 = __ldg(T.halo_off + t);
      unsigned char* buf = sm + (size_t)b * L.buf;
      if (lane == 0)
        mbar_arrive_tx(&full[b], (uint32_t)((Pt + nh) * kHW * sizeof(float) +
                                            (size_t)ne * (sizeof(uint16_t) + sizeof(float))));
      __syncwarp();
      if (lane == 0) {
        bulk_copy(buf + L.idx, T.ell_idx + e0, (uint32_t)(ne * sizeof(uint16_t)), &full[b]);
        bulk_copy(buf + L.val, T.ell_val + e0, (uint32_t)(ne * sizeof(float)), &full[b]);
      }
      const float* src = a.p + a.col0 + ch * kHW;
      // the halo row ids of a batch are loaded together, then copied
      for (int j0 = 0; j0 < Pt + nh; j0 += 32 * kBatch) {
        int64_t gs[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int j = j0 + 32 * u + lane;
          gs[u] = j < Pt ? t0 + j : j < Pt + nh ? (int64_t)__ldg(T.halo + h0 + (j - Pt)) : -1;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int j = j0 + 32 * u + lane;
          if (gs[u] >= 0)
            bulk_copy(buf + (size_t)j * kHW * sizeof(float), src + gs[u] * a.ld,
                      kHW * sizeof(float), &full[b]);
        }
      }
      issued = i + 1;
    }
    // copies in flight land before the CTA may leave (bounded)
    for (int i = max(0, issued - 2); i < issued; ++i) mbar_wait(&full[i & 1], (i >> 1) & 1);
    return;
  }

  // -------------------------------------------------------------- consumers
  const int g = lane / kLPR, lr = lane % kLPR;
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  for (int i = 0; i < n_items; ++i) {
    const int b = i & 1;
    if (!mbar_wait(&full[b], (uint32_t)(i >> 1) & 1)) {
      atomicExch(err, 1);
      return;
    }
    const int t = t_begin + i / nchunk, ch = i % nchunk;
    const int64_t t0 = (int64_t)t * T.P;
    const int Pt = (int)(n - t0 < (int64_t)T.P ? n - t0 : (int64_t)T.P);
    const unsigned char* buf = sm + (size_t)b * L.buf;
    const float4* rows = reinterpret_cast<const float4*>(buf);
    const uint16_t* idx = reinterpret_cast<const uint16_t*>(buf + L.idx);
    const float* val = reinterpret_cast<const float*>(buf + L.val);
    const int col0 = a.col0 + ch * kHW;
    for (int rl = warp * kRPW + g; rl < Pt; rl += kRPP) {
      const int64_t row = t0 + rl;
      const size_t ro = (size_t)row * a.ld + col0 + 4 * lr;
      const int s0 = __ldg(a.ev.src_ptr + row), s1 = __ldg(a.ev.src_ptr + row + 1);
      const float4 old = *reinterpret_cast<const float4*>(a.pm + ro);
      const float4 c = __ldg(a.coef + row);
      const int2 si = __ldg(reinterpret_cast<const int2*>(T.slice_info) + row / kSliceH);
      const int rs = (int)(row % kSliceH);
      const uint16_t* ix = idx + si.x + rs;
      const float* vv = val + si.x + rs;
      const float4 self = rows[(size_t)rl * kLPR + lr];
      float4 acc = scale4(vv[0], self);
#pragma unroll 4
      for (int k = 1; k < si.y; ++k)
        acc = fma4(vv[k * kSliceH], rows[(size_t)ix[k * kSliceH] * kLPR + lr], acc);
      float4 out = leap(c, self, old, acc);
      if (s0 != s1) {
        const float sv = c.z * __ldg(a.wavelet + l);
        for (int q = s0; q < s1; ++q) {
          int d;
          if (mine(__ldg(a.ev.src_shot + q), col0, lr, d)) add_comp(out, d, sv);
        }
      }
      st4(a.pout + ro, out);
      if (a.traces) {
        const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
        for (int q = r0; q < r1; ++q) {
          int d;
          if (mine(__ldg(a.ev.rec_shot + q), col0, lr, d))
            a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = get_comp(out, d);
        }
      }
    }
    fence_async_shared();                           // reads before the next copies into b
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[b]);
  }
}

}  // namespace

size_t tma_smem_bytes(const DevTiles& T) { return tma_layout(T).total; }

int launch_step_tma(const StepArgs& a, const DevTiles& T, int S_pad, int* err, cudaStream_t st) {
  const int cols = a.cols ? a.cols : S_pad;
  if (!err || T.P <= 0 || T.P % kSliceH || T.n_tiles < 1 || cols % kHW || a.col0 % kHW ||
      a.col0 < 0 || a.col0 + cols > a.ld || a.ld % 4)
    return cols % kHW || a.col0 % kHW ? MG_ERR_UNSUPPORTED : MG_ERR_ARG;
  const size_t smem = tma_smem_bytes(T);
  int dev = 0, nsm = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  if (smem > (size_t)optin) return MG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_step_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  const int grid = std::min(T.n_tiles, nsm);         // one CTA per SM (shared memory)
  const int per = (T.n_tiles + grid - 1) / grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((T.n_tiles + per - 1) / per);
  cfg.blockDim = dim3(kTmaThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = a.pdl ? 1 : 0;
  if (cudaLaunchKernelEx(&cfg, k_step_tma, a, T, err, per) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  return check_launch();
}

}  // namespace mg
