// Forward leapfrog step with the neighbour rows staged in shared memory by
// bulk asynchronous copies (cp.async.bulk, the TMA engine) completing on a
// per-warp mbarrier.
//
// Layout and arithmetic are those of the row kernels (kernels_rows.cu): LPR
// lanes per row, NV float4 of shots per lane, the row's stiffness entries
// read LPR at a time (one per lane) and handed out by shuffles, the same
// accumulation order, so the results carry the same bits.  What changes is
// how the neighbour values arrive: for a chunk of LPR entries every lane
// issues one bulk copy of its entry's segment of the neighbour row (the
// 4*LPR*NV shots of the source tile, 16*LPR*NV bytes, 16-byte aligned) into
// the warp's slot of shared memory, so all neighbours of the chunk are in
// flight at once without holding registers; the warp then waits on its
// mbarrier (bounded: on time-out it records an error, waits once more for
// its copies, and leaves) and accumulates from shared memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mgwave.h"
#include "device_util.cuh"
#include "kernels.cuh"
#include "mg_internal.h"
#include "async_copy.cuh"

namespace mg {
namespace {

using namespace dev;

constexpr int kBulkWarps = 4;
constexpr int kBulkThreads = 32 * kBulkWarps;

using namespace ac;

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  ac::mbar_init(bar, 1);
  mbar_init_fence();
}

__device__ __forceinline__ int2 entry_at(const int2* e, int w, int k, int row) {
  return k < w ? __ldg(e + (size_t)k * kSliceH) : make_int2(row, 0);
}

// Dynamic shared memory: per warp RPW * LPR slots of TW floats, then the
// warps' mbarriers.
template <int LPR, int NV>
__global__ void __launch_bounds__(kBulkThreads) k_step_bulk(StepArgs a, int* err) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  extern __shared__ __align__(128) float sbuf[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* slots = sbuf + (size_t)warp * RPW * LPR * TW;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sbuf + (size_t)kBulkWarps * RPW * LPR * TW) + warp;
  const int row0 = (blockIdx.x * kBulkWarps + warp) * RPW;
  if (row0 >= a.K.n) return;                          // whole warp leaves together
  const int g = lane / LPR, lr = lane % LPR;
  const int row = row0 + g;
  const bool valid = row < a.K.n;
  const unsigned mask = __ballot_sync(0xffffffffu, valid);
  if (lane == 0) mbar_init(bar);
  __syncwarp();
  const int tile0 = a.col0 + blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  const int slice = row0 / kSliceH;
  const int2* e = a.K.ell + __ldg(a.K.slice_off + slice) + (row0 - slice * kSliceH) + g;
  const int w = __ldg(a.K.slice_w + slice);
  float4 old[NV], self[NV], acc[NV];
  const size_t ro = (size_t)(valid ? row : row0) * a.ld + base;
#pragma unroll
  for (int j = 0; j < NV; ++j) old[j] = *reinterpret_cast<const float4*>(a.pm + ro + 4 * LPR * j);
  float* myslot = slots + (size_t)(g * LPR) * TW;   // this row's LPR slots
  uint32_t parity = 0;
  float v0 = 0.0f;
  const uint32_t bytes = TW * sizeof(float);
  for (int k0 = 0; k0 < w; k0 += LPR) {
    const int2 ent = entry_at(e, w, k0 + lr, row);
    const float* src = a.p + (size_t)ent.x * a.ld + tile0;
    float* dst = myslot + (size_t)lr * TW;
    const bool want = valid && k0 + lr < w;
    // 16-byte alignment holds for every launch shape (ld and tile0 are
    // multiples of 4 floats); a violation is recorded and the copy skipped,
    // which leaves the phase incomplete and ends the wait below with an error
    const bool aligned = ((reinterpret_cast<uintptr_t>(src) | s_addr(dst)) & 15u) == 0;
    if (want && !aligned) atomicExch(err, 2);
    // the phase expects every wanted segment; lane 0 arrives before any copy
    const int n_want = __popc(__ballot_sync(0xffffffffu, want));
    if (lane == 0) mbar_arrive_tx(bar, (uint32_t)n_want * bytes);
    __syncwarp();
    if (want && aligned) bulk_copy(dst, src, bytes, bar);
    const bool done = __all_sync(0xffffffffu, mbar_wait(bar, parity));
    if (!done) {                                      // uniform across the warp
      if (lane == 0) atomicExch(err, 1);
      mbar_wait(bar, parity);                         // let copies in flight land
      return;
    }
    parity ^= 1u;
    if (valid) {
      const int kn = min(LPR, w - k0);
      for (int k = 0; k < kn; ++k) {
        const float v = __int_as_float(__shfl_sync(mask, ent.y, k, LPR));
        const float* xs = myslot + (size_t)k * TW + 4 * lr;
        if (k0 == 0 && k == 0) {
          v0 = v;
#pragma unroll
          for (int j = 0; j < NV; ++j) {
            self[j] = *reinterpret_cast<const float4*>(xs + 4 * LPR * j);
            acc[j] = scale4(v0, self[j]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < NV; ++j)
            acc[j] = fma4(v, *reinterpret_cast<const float4*>(xs + 4 * LPR * j), acc[j]);
        }
      }
    }
    fence_async_shared();
    __syncwarp();
  }
  if (!valid) return;
  const float4 c = __ldg(a.coef + row);
  float4 out[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = leap(c, self[j], old[j], acc[j]);
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  const int s0 = __ldg(a.ev.src_ptr + row), s1 = __ldg(a.ev.src_ptr + row + 1);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      const int rel = __ldg(a.ev.src_shot + q) - tile0;
      if (rel < 0 || rel >= TW) continue;
      const int within = rel % (4 * LPR);
      if (within / 4 != lr) continue;
      const int j = rel / (4 * LPR), d = within % 4;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i == j) add_comp(out[i], d, sv);
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) st4(a.pout + ro + 4 * LPR * j, out[j]);
  if (a.traces) {
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      const int rel = __ldg(a.ev.rec_shot + q) - tile0;
      if (rel < 0 || rel >= TW) continue;
      const int within = rel % (4 * LPR);
      if (within / 4 != lr) continue;
      const int j = rel / (4 * LPR), d = within % 4;
      float v = 0.0f;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i == j) v = get_comp(out[i], d);
      a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = v;
    }
  }
}

template <int LPR, int NV>
int launch_bulk(const StepArgs& a, int cols, int* err, cudaStream_t st) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const size_t smem = (size_t)kBulkWarps * RPW * LPR * TW * sizeof(float) +
                      kBulkWarps * sizeof(uint64_t);
  if (cudaFuncSetAttribute(k_step_bulk<LPR, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  const int rows_per_block = kBulkWarps * RPW;
  const dim3 grid((a.K.n + rows_per_block - 1) / rows_per_block, cols / TW);
  k_step_bulk<LPR, NV><<<grid, kBulkThreads, smem, st>>>(a, err);
  return check_launch();
}

}  // namespace

// Forward step with bulk-copied neighbour rows; shapes as launch_step (LPR
// lanes per row chosen from the column count, NV = min(a.batch, 2)).
int launch_step_bulk(const StepArgs& a, int S_pad, int* err, cudaStream_t st) {
  const int cols = a.cols ? a.cols : S_pad;
  int nv = a.batch > 2 ? 2 : a.batch;   // variants for 1 and 2 float4 per lane
  int lpr = 0;
  for (;; nv >>= 1) {
    lpr = cols / (4 * nv) >= 32 ? 32 : cols / (4 * nv);
    if (nv == 1 || (lpr >= 1 && (lpr & (lpr - 1)) == 0 && cols % (4 * nv * lpr) == 0)) break;
  }
  const int tw = 4 * nv * lpr;
  if (lpr < 1 || a.col0 < 0 || a.col0 % tw || cols % tw || a.col0 + cols > a.ld || !err)
    return MG_ERR_ARG;
  switch (lpr * 8 + nv) {
    case 32 * 8 + 1: return launch_bulk<32, 1>(a, cols, err, st);
    case 32 * 8 + 2: return launch_bulk<32, 2>(a, cols, err, st);
    case 16 * 8 + 1: return launch_bulk<16, 1>(a, cols, err, st);
    case 16 * 8 + 2: return launch_bulk<16, 2>(a, cols, err, st);
    case 8 * 8 + 1: return launch_bulk<8, 1>(a, cols, err, st);
    case 8 * 8 + 2: return launch_bulk<8, 2>(a, cols, err, st);
    case 4 * 8 + 1: return launch_bulk<4, 1>(a, cols, err, st);
    case 4 * 8 + 2: return launch_bulk<4, 2>(a, cols, err, st);
    case 2 * 8 + 1: return launch_bulk<2, 1>(a, cols, err, st);
    case 2 * 8 + 2: return launch_bulk<2, 2>(a, cols, err, st);
    case 1 * 8 + 1: return launch_bulk<1, 1>(a, cols, err, st);
    case 1 * 8 + 2: return launch_bulk<1, 2>(a, cols, err, st);
    default: return MG_ERR_UNSUPPORTED;
  }
}

}  // namespace mg
