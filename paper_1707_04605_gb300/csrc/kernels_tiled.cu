// Shared-memory tiled leapfrog kernels (sm_103a).
//
// One CTA per row tile (HostTiles).  Phase 0 stages, once per launch, the
// tile's slice table, its stiffness entries with 16-bit local indices, its
// halo list, the per-row coefficients and the per-row source/receiver list
// pointers.  The shots are then processed in passes of ST: for each pass
// the state rows of the tile and of its halo (the rows its neighbours live
// in) and the tile's own rows of every other state the step reads are
// copied into shared memory with 16-byte cp.async, double buffered so that
// pass s+1 streams in while pass s is computed.  The compute phase reads
// only shared memory and writes results with coalesced stores, so the
// number of resident warps no longer bounds the memory parallelism.
#include <cuda_runtime.h>

#include "../../include/mgwave.h"
#include "device_util.cuh"
#include "kernels.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

using namespace dev;

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// Shared-memory layout of one CTA.  `halo_states` states are staged for the
// tile and its halo (they are gathered through the stencil); `row_states`
// for the tile's own rows only.
struct Layout {
  size_t sinfo, idx, val, halo, coef, srcp, recp, buf, pass_bytes, total;
};

__host__ __device__ __forceinline__ Layout layout(const DevTiles& T, int halo_states,
                                                  int row_states, int coef_floats) {
  Layout L;
  size_t o = 0;
  L.sinfo = o; o += al16((size_t)(T.P / kSliceH) * 8);
  L.idx = o;   o += al16((size_t)T.max_ell * 2);
  L.val = o;   o += al16((size_t)T.max_ell * 4);
  L.halo = o;  o += al16((size_t)T.max_halo * 4);
  L.coef = o;  o += al16((size_t)T.P * coef_floats * 4);
  L.srcp = o;  o += al16((size_t)(T.P + 1) * 4);
  L.recp = o;  o += al16((size_t)(T.P + 1) * 4);
  L.buf = o;
  L.pass_bytes = ((size_t)halo_states * (T.P + T.max_halo) + (size_t)row_states * T.P) *
                 T.st_w * sizeof(float);
  o += 2 * L.pass_bytes;
  L.total = o;
  return L;
}

struct Tile {
  int t;
  int64_t t0;
  int Pt;      // own rows
  int nrows;   // own + halo rows
};

// Phase 0: tables of the tile (one cp.async group, waited for here).
__device__ __forceinline__ Tile stage_tables(const DevTiles& T, const Layout& L,
                                             unsigned char* sm, int64_t n, const float4* coef,
                                             const float2* coef2, const DevEvents& ev,
                                             bool want_rec) {
  Tile tl;
  tl.t = blockIdx.x;
  tl.t0 = (int64_t)tl.t * T.P;
  tl.Pt = (int)(n - tl.t0 < T.P ? n - tl.t0 : T.P);
  const int spt = (tl.Pt + kSliceH - 1) / kSliceH;
  const int tid = threadIdx.x, nth = blockDim.x;
  int2* sinfo = reinterpret_cast<int2*>(sm + L.sinfo);
  for (int i = tid; i < spt; i += nth) cp8(sinfo + i, T.slice_info + 2 * (tl.t0 / kSliceH + i));
  const int64_t e0 = T.ell_off[tl.t];
  const int ne = (int)(T.ell_off[tl.t + 1] - e0);
  uint16_t* idx = reinterpret_cast<uint16_t*>(sm + L.idx);
  float* val = reinterpret_cast<float*>(sm + L.val);
  for (int c = tid; c < ne / 8; c += nth) cp16(idx + 8 * c, T.ell_idx + e0 + 8 * c);
  for (int c = tid; c < ne / 4; c += nth) cp16(val + 4 * c, T.ell_val + e0 + 4 * c);
  const int64_t h0 = T.halo_off[tl.t];
  const int nh = (int)(T.halo_off[tl.t + 1] - h0);
  int32_t* halo = reinterpret_cast<int32_t*>(sm + L.halo);
  for (int c = tid; c < nh / 4; c += nth) cp16(halo + 4 * c, T.halo + h0 + 4 * c);
  float4* sc = reinterpret_cast<float4*>(sm + L.coef);
  for (int i = tid; i < tl.Pt; i += nth) cp16(sc + i, coef + tl.t0 + i);
  if (coef2) {
    float2* sc2 = reinterpret_cast<float2*>(sm + L.coef + (size_t)T.P * 16);
    for (int i = tid; i < tl.Pt; i += nth) cp8(sc2 + i, coef2 + tl.t0 + i);
  }
  int32_t* sp = reinterpret_cast<int32_t*>(sm + L.srcp);
  int32_t* rp = reinterpret_cast<int32_t*>(sm + L.recp);
  for (int i = tid; i <= tl.Pt; i += nth) {
    cp4(sp + i, ev.src_ptr + tl.t0 + i);
    if (want_rec) cp4(rp + i, ev.rec_ptr + tl.t0 + i);
  }
  cp_commit();
  cp_wait<0>();
  __syncthreads();
  tl.nrows = tl.Pt + T.halo_cnt[tl.t];
  return tl;
}

// Copies the ST shots of pass `st` of the rows [0, nrows) (own rows, then
// halo rows) of `src` into `dst` ([nrows][ST]).
template <int ST>
__device__ __forceinline__ void stage_rows(const Tile& tl, const int32_t* halo, int nrows,
                                           const float* __restrict__ src, int ld, int st,
                                           float* dst) {
  constexpr int CPR = ST / 4;
  for (int c = threadIdx.x; c < nrows * CPR; c += blockDim.x) {
    const int r = c / CPR, part = c - r * CPR;
    const int64_t g = r < tl.Pt ? tl.t0 + r : (int64_t)halo[r - tl.Pt];
    cp16(dst + (size_t)r * ST + part * 4, src + (size_t)g * ld + (size_t)st * ST + part * 4);
  }
}

// Stencil sum over the row's local entries (diagonal first) from `buf`.
template <int ST>
__device__ __forceinline__ float4 row_acc(const int2* sinfo, const uint16_t* idx,
                                          const float* val, const float* buf, int li, int lr,
                                          float4& self) {
  const int2 si = sinfo[li / kSliceH];
  const int rl = li % kSliceH;
  self = *reinterpret_cast<const float4*>(buf + (size_t)li * ST + lr * 4);
  float4 acc = scale4(val[si.x + rl], self);
  for (int k = 1; k < si.y; ++k) {
    const int o = si.x + k * kSliceH + rl;
    acc = fma4(val[o], *reinterpret_cast<const float4*>(buf + (size_t)idx[o] * ST + lr * 4), acc);
  }
  return acc;
}

template <int ST>
__device__ __forceinline__ void row_acc2(const int2* sinfo, const uint16_t* idx, const float* val,
                                         const float* bp, const float* bq, int li, int lr,
                                         float4& ps, float4& qs, float4& pacc, float4& qacc) {
  const int2 si = sinfo[li / kSliceH];
  const int rl = li % kSliceH;
  ps = *reinterpret_cast<const float4*>(bp + (size_t)li * ST + lr * 4);
  qs = *reinterpret_cast<const float4*>(bq + (size_t)li * ST + lr * 4);
  const float v0 = val[si.x + rl];
  pacc = scale4(v0, ps);
  qacc = scale4(v0, qs);
  for (int k = 1; k < si.y; ++k) {
    const int o = si.x + k * kSliceH + rl;
    const size_t off = (size_t)idx[o] * ST + lr * 4;
    const float v = val[o];
    pacc = fma4(v, *reinterpret_cast<const float4*>(bp + off), pacc);
    qacc = fma4(v, *reinterpret_cast<const float4*>(bq + off), qacc);
  }
}

constexpr int kTWarps = 8;
constexpr int kTThreads = 32 * kTWarps;

// Pass buffer b: halo-staged state(s) first, then the row-only states.
#define PASS_BUF(b) reinterpret_cast<float*>(smem + L.buf + (size_t)(b) * L.pass_bytes)

template <int ST>
__global__ void __launch_bounds__(kTThreads) k_step_tiled(StepArgs a, DevTiles T) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int LPR = ST / 4, RPW = 32 / LPR;
  const Layout L = layout(T, 1, 1, 4);
  const Tile tl = stage_tables(T, L, smem, a.K.n, a.coef, nullptr, a.ev, a.traces != nullptr);
  const int2* sinfo = reinterpret_cast<const int2*>(smem + L.sinfo);
  const uint16_t* idx = reinterpret_cast<const uint16_t*>(smem + L.idx);
  const float* val = reinterpret_cast<const float*>(smem + L.val);
  const int32_t* halo = reinterpret_cast<const int32_t*>(smem + L.halo);
  const float4* sc = reinterpret_cast<const float4*>(smem + L.coef);
  const int32_t* sp = reinterpret_cast<const int32_t*>(smem + L.srcp);
  const int32_t* rp = reinterpret_cast<const int32_t*>(smem + L.recp);
  const size_t hrows = (size_t)(T.P + T.max_halo) * ST;  // offset of the row-only state
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lr = lane % LPR;
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  const int NST = (a.cols ? a.cols : a.ld) / ST;
  auto issue = [&](int st) {
    float* b = PASS_BUF(st & 1);
    stage_rows<ST>(tl, halo, tl.nrows, a.p + a.col0, a.ld, st, b);
    stage_rows<ST>(tl, halo, tl.Pt, a.pm + a.col0, a.ld, st, b + hrows);
    cp_commit();
  };
  issue(0);
  for (int st = 0; st < NST; ++st) {
    if (st + 1 < NST) {
      issue(st + 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const float* cur = PASS_BUF(st & 1);
    const float* pmr = cur + hrows;
    const int src0 = a.col0 + st * ST + lr * 4;
    for (int li = warp * RPW + lane / LPR; li < tl.Pt; li += kTWarps * RPW) {
      float4 self;
      const float4 acc = row_acc<ST>(sinfo, idx, val, cur, li, lr, self);
      const float4 old = *reinterpret_cast<const float4*>(pmr + (size_t)li * ST + lr * 4);
      const float4 c = sc[li];
      float4 out = leap(c, self, old, acc);
      const int64_t row = tl.t0 + li;
      const int s0 = sp[li], s1 = sp[li + 1];
      if (s0 != s1) {
        const float sv = c.z * __ldg(a.wavelet + l);
        for (int q = s0; q < s1; ++q) {
          const int d = __ldg(a.ev.src_shot + q) - src0;
          if (d >= 0 && d < 4) add_comp(out, d, sv);
        }
      }
      st4(a.pout + (size_t)row * a.ld + src0, out);
      if (a.traces) {
        const int r0 = rp[li], r1 = rp[li + 1];
        for (int q = r0; q < r1; ++q) {
          const int d = __ldg(a.ev.rec_shot + q) - src0;
          if (d >= 0 && d < 4)
            a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = get_comp(out, d);
        }
      }
    }
    __syncthreads();
  }
}

template <int ST>
__global__ void __launch_bounds__(kTThreads) k_tangent_tiled(TangentArgs a, DevTiles T) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int LPR = ST / 4, RPW = 32 / LPR;
  const Layout L = layout(T, 2, 2, 6);
  const Tile tl = stage_tables(T, L, smem, a.f.K.n, a.f.coef, a.tcoef, a.f.ev, true);
  const int2* sinfo = reinterpret_cast<const int2*>(smem + L.sinfo);
  const uint16_t* idx = reinterpret_cast<const uint16_t*>(smem + L.idx);
  const float* val = reinterpret_cast<const float*>(smem + L.val);
  const int32_t* halo = reinterpret_cast<const int32_t*>(smem + L.halo);
  const float4* sc = reinterpret_cast<const float4*>(smem + L.coef);
  const float2* sc2 = reinterpret_cast<const float2*>(smem + L.coef + (size_t)T.P * 16);
  const int32_t* sp = reinterpret_cast<const int32_t*>(smem + L.srcp);
  const int32_t* rp = reinterpret_cast<const int32_t*>(smem + L.recp);
  const size_t hrows = (size_t)(T.P + T.max_halo) * ST;
  const size_t prow = (size_t)T.P * ST;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lr = lane % LPR;
  const int ld = a.f.ld;
  const int l = a.f.step + (a.f.step_base ? *a.f.step_base : 0);
  const int c0 = a.f.col0;
  const int NST = (a.f.cols ? a.f.cols : ld) / ST;
  // pass buffer: [p rows+halo][q rows+halo][p_{l-1} rows][q_{l-1} rows]
  auto issue = [&](int st) {
    float* b = PASS_BUF(st & 1);
    stage_rows<ST>(tl, halo, tl.nrows, a.f.p + c0, ld, st, b);
    stage_rows<ST>(tl, halo, tl.nrows, a.q + c0, ld, st, b + hrows);
    stage_rows<ST>(tl, halo, tl.Pt, a.f.pm + c0, ld, st, b + 2 * hrows);
    stage_rows<ST>(tl, halo, tl.Pt, a.qm + c0, ld, st, b + 2 * hrows + prow);
    cp_commit();
  };
  issue(0);
  for (int st = 0; st < NST; ++st) {
    if (st + 1 < NST) {
      issue(st + 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const float* bp = PASS_BUF(st & 1);
    const float* bq = bp + hrows;
    const float* bpm = bp + 2 * hrows;
    const float* bqm = bpm + prow;
    const int src0 = c0 + st * ST + lr * 4;
    for (int li = warp * RPW + lane / LPR; li < tl.Pt; li += kTWarps * RPW) {
      float4 ps, qs, acc, qacc;
      row_acc2<ST>(sinfo, idx, val, bp, bq, li, lr, ps, qs, acc, qacc);
      const float4 pold = *reinterpret_cast<const float4*>(bpm + (size_t)li * ST + lr * 4);
      const float4 qold = *reinterpret_cast<const float4*>(bqm + (size_t)li * ST + lr * 4);
      const float4 c = sc[li];
      const float2 tc = sc2[li];
      const int64_t row = tl.t0 + li;
      float4 pn = leap(c, ps, pold, acc);
      const int s0 = sp[li], s1 = sp[li + 1];
      if (s0 != s1) {
        const float sv = c.z * __ldg(a.f.wavelet + l);
        for (int q = s0; q < s1; ++q) {
          const int d = __ldg(a.f.ev.src_shot + q) - src0;
          if (d >= 0 && d < 4) add_comp(pn, d, sv);
        }
      }
      // dp+ = alpha dp - beta dp- - gamma K dp - cm (p+ - 2p + p-) - cd (p+ - p-)
      const float4 qn = tangent_fix(leap(c, qs, qold, qacc), pn, ps, pold, tc);
      const size_t ro = (size_t)row * ld + src0;
      st4(a.f.pout + ro, pn);
      st4(a.qm + ro, qn);
      const int r0 = rp[li], r1 = rp[li + 1];
      for (int q = r0; q < r1; ++q) {
        const int d = __ldg(a.f.ev.rec_shot + q) - src0;
        if (d >= 0 && d < 4)
          a.dtraces[(size_t)__ldg(a.f.ev.rec_trace + q) * a.f.nt + l] = get_comp(qn, d);
      }
    }
    __syncthreads();
  }
}

template <int ST>
__global__ void __launch_bounds__(kTThreads) k_adjoint_tiled(AdjointArgs a, DevTiles T) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int LPR = ST / 4, RPW = 32 / LPR;
  const Layout L = layout(T, 1, 2, 4);
  // per-row partial sums over all shots, after the pass buffers
  float* t1s = reinterpret_cast<float*>(smem + L.total);
  float* t2s = t1s + T.P;
  for (int i = threadIdx.x; i < T.P; i += blockDim.x) { t1s[i] = 0.0f; t2s[i] = 0.0f; }
  const Tile tl = stage_tables(T, L, smem, a.K.n, a.coef, nullptr, a.ev, true);
  const int2* sinfo = reinterpret_cast<const int2*>(smem + L.sinfo);
  const uint16_t* idx = reinterpret_cast<const uint16_t*>(smem + L.idx);
  const float* val = reinterpret_cast<const float*>(smem + L.val);
  const int32_t* halo = reinterpret_cast<const int32_t*>(smem + L.halo);
  const float4* sc = reinterpret_cast<const float4*>(smem + L.coef);
  const int32_t* rp = reinterpret_cast<const int32_t*>(smem + L.recp);
  const size_t hrows = (size_t)(T.P + T.max_halo) * ST;
  const size_t prow = (size_t)T.P * ST;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lr = lane % LPR;
  const int k = a.k + (a.step_base ? *a.step_base : 0);
  const int NST = (a.cols ? a.cols : a.ld) / ST;
  // pass buffer: [mu_k rows+halo][mu_{k+1} rows][p_k rows]
  auto issue = [&](int st) {
    float* b = PASS_BUF(st & 1);
    stage_rows<ST>(tl, halo, tl.nrows, a.mu + a.col0, a.ld, st, b);
    stage_rows<ST>(tl, halo, tl.Pt, a.mu1 + a.col0, a.ld, st, b + hrows);
    stage_rows<ST>(tl, halo, tl.Pt, a.pk + a.col0, a.ld, st, b + hrows + prow);
    cp_commit();
  };
  issue(0);
  for (int st = 0; st < NST; ++st) {
    if (st + 1 < NST) {
      issue(st + 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const float* cur = PASS_BUF(st & 1);
    const float* b1 = cur + hrows;
    const float* bk = b1 + prow;
    const int src0 = a.col0 + st * ST + lr * 4;
    for (int base = 0; base < tl.Pt; base += kTWarps * RPW) {
      const int li = base + warp * RPW + lane / LPR;
      float t1 = 0.0f, t2 = 0.0f;
      if (li < tl.Pt) {
        float4 self;
        const float4 acc = row_acc<ST>(sinfo, idx, val, cur, li, lr, self);
        const float4 old = *reinterpret_cast<const float4*>(b1 + (size_t)li * ST + lr * 4);
        const float4 pk = *reinterpret_cast<const float4*>(bk + (size_t)li * ST + lr * 4);
        const float4 c = sc[li];
        float4 out = leap(c, self, old, acc);
        const int r0 = rp[li], r1 = rp[li + 1];
        for (int q = r0; q < r1; ++q) {
          const int d = __ldg(a.ev.rec_shot + q) - src0;
          if (d >= 0 && d < 4)
            add_comp(out, d, c.w * __ldg(a.w + (size_t)__ldg(a.ev.rec_trace + q) * a.nt + (k - 1)));
        }
        st4(a.mu1 + (size_t)(tl.t0 + li) * a.ld + src0, out);
        adj_terms(pk, out, self, old, t1, t2);
      }
#pragma unroll
      for (int off = LPR / 2; off > 0; off >>= 1) {
        t1 += __shfl_xor_sync(0xffffffffu, t1, off);
        t2 += __shfl_xor_sync(0xffffffffu, t2, off);
      }
      if (li < tl.Pt && lr == 0) {
        t1s[li] += t1;
        t2s[li] += t2;
      }
    }
    __syncthreads();
  }
  for (int li = threadIdx.x; li < tl.Pt; li += blockDim.x) {
    const size_t gi = (size_t)(tl.t0 + li);
    kahan_add(a.G + gi, a.Gc + gi, t1s[li]);
    kahan_add(a.H + gi, a.Hc + gi, t2s[li]);
  }
}
#undef PASS_BUF

template <class K>
int prepare_launch(K kern, size_t smem) {
  static int optin = -1;
  if (optin < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return MG_ERR_CUDA;
  }
  if (smem > (size_t)optin) return MG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return MG_ERR_CUDA;
  }
  return MG_OK;
}

}  // namespace

size_t tiled_smem_bytes(const DevTiles& T, int kind) {
  switch (kind) {
    case 0: return layout(T, 1, 1, 4).total;                                  // forward
    case 1: return layout(T, 2, 2, 6).total;                                  // tangent
    default: return layout(T, 1, 2, 4).total + 2 * (size_t)T.P * sizeof(float);  // adjoint
  }
}

#define MG_TILED_CASE(KERN, W, ARGS, SMEM)                                            \
  case W:                                                                             \
    rc = prepare_launch(KERN<W>, SMEM);                                               \
    if (!rc) KERN<W><<<T.n_tiles, kTThreads, SMEM, st>>>(ARGS, T);                    \
    break;
#define MG_TILED_SWITCH(KERN, ARGS, SMEM)                                             \
  switch (T.st_w) {                                                                   \
    MG_TILED_CASE(KERN, 4, ARGS, SMEM) MG_TILED_CASE(KERN, 8, ARGS, SMEM)             \
    MG_TILED_CASE(KERN, 16, ARGS, SMEM) MG_TILED_CASE(KERN, 32, ARGS, SMEM)           \
    MG_TILED_CASE(KERN, 64, ARGS, SMEM)                                               \
    default: return MG_ERR_ARG;                                                       \
  }

// The passes cover shot columns [col0, col0 + cols): whole passes of st_w
// shots inside ld, starting on a 16-byte boundary.
bool tiled_range_ok(int col0, int cols, int ld, int st_w) {
  if (!cols) cols = ld;
  return col0 >= 0 && col0 % 4 == 0 && cols > 0 && col0 + cols <= ld && cols % st_w == 0;
}

int launch_step_tiled(const StepArgs& a, const DevTiles& T, cudaStream_t st) {
  if (!tiled_range_ok(a.col0, a.cols, a.ld, T.st_w)) return MG_ERR_ARG;
  int rc = MG_OK;
  const size_t smem = tiled_smem_bytes(T, 0);
  MG_TILED_SWITCH(k_step_tiled, a, smem)
  return rc ? rc : check_launch();
}

int launch_tangent_tiled(const TangentArgs& a, const DevTiles& T, cudaStream_t st) {
  if (!tiled_range_ok(a.f.col0, a.f.cols, a.f.ld, T.st_w)) return MG_ERR_ARG;
  int rc = MG_OK;
  const size_t smem = tiled_smem_bytes(T, 1);
  MG_TILED_SWITCH(k_tangent_tiled, a, smem)
  return rc ? rc : check_launch();
}

int launch_adjoint_tiled(const AdjointArgs& a, const DevTiles& T, cudaStream_t st) {
  if (!tiled_range_ok(a.col0, a.cols, a.ld, T.st_w)) return MG_ERR_ARG;
  int rc = MG_OK;
  const size_t smem = tiled_smem_bytes(T, 2);
  MG_TILED_SWITCH(k_adjoint_tiled, a, smem)
  return rc ? rc : check_launch();
}
#undef MG_TILED_SWITCH
#undef MG_TILED_CASE

}  // namespace mg
