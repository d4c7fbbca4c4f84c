// Row-parallel (untiled) leapfrog kernels: forward step, forward+tangent
// step and reverse adjoint step, for every shot of a batch.  Included by
// kernels_rows.cu (plain gathers) and kernels_ring.cu (gathers pipelined
// through a shared-memory ring), which instantiate and launch them.
//
// State layout: node-major [row][ld] FP32, ld = padded shot count.  A lane
// carries NV float4 (4*NV shots); LPR lanes cover a source tile of
// TW = 4*NV*LPR shots of one row, so a warp advances 32/LPR rows.  The
// lane's j-th float4 holds shots base + 4*LPR*j .. +3, so every vector load
// of the LPR lanes of a row reads one contiguous 16*LPR-byte span.
// The stiffness entries (col, K) of a row are loaded once per row and
// handed to its LPR lanes by shuffles; each serves the 4*NV shots of a lane.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

#include "../../include/mgwave.h"
#include "device_util.cuh"
#include "kernels.cuh"
#include "mg_internal.h"

namespace mg {
namespace {

using namespace dev;

// Programmatic dependent launch: wait until the kernel this launch depends
// on has completed and its writes are visible (a no-op for a launch that was
// not made dependent), then let the next dependent launch start.  Everything
// a kernel does before this call reads only the stiffness slice table, which
// no step writes.
__device__ __forceinline__ void grid_dep_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Load of a row's float4 that is its state's last use in this pass: with
// an L2 evict-first policy when `hint` is set (the kept history streams
// more states than L2 holds; the lines still to be read are kept instead),
// and without L1 allocation when `na` is set (L1 keeps the neighbour rows
// the gathers reuse).  NC: read-only data of the launch (no store of this
// launch aliases it); otherwise the load is a memory access the compiler
// keeps in place (the same thread may overwrite the data later).
template <bool NC>
__device__ __forceinline__ float4 ld_once(const float* p, int hint, int na) {
  float4 v;
  if (!hint && !na)
    return NC ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
  if (!hint) {
    if (NC)
      asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                   : "l"(p));
    else
      asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                   : "l"(p)
                   : "memory");
    return v;
  }
  if (na)
    asm volatile(
        "{\n\t.reg .b64 pol;\n\t"
        "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
        "ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], pol;\n\t}"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .b64 pol;\n\t"
        "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
        "ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], pol;\n\t}"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p)
        : "memory");
  return v;
}

struct Row {
  const int2* e;  // entry 0 of the row (stride kSliceH)
  int w;          // entries of the row's slice, diagonal first
  int na = 0;     // load the entries without allocating them in L1
};

// Read-only per-row data (coefficients, stiffness entries) loaded once per
// launch, without L1 allocation when `na` is set.
__device__ __forceinline__ float4 ldg_stream4(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ int2 ldg_stream2(const int2* p) {
  int2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.s32 {%0, %1}, [%2];"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ldg_stream2f(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];"
               : "=f"(v.x), "=f"(v.y)
               : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_coef(const float4* p, int na) {
  return na ? ldg_stream4(p) : __ldg(p);
}
__device__ __forceinline__ float2 ld_coef(const float2* p, int na) {
  return na ? ldg_stream2f(p) : __ldg(p);
}

// The row as lane lr of its LPR lanes sees it: e points at the lane's entry
// of the row's first chunk of LPR entries; the chunk starting at entry k0
// lies 32 k0 entries further in both layouts.  By column (sliced or, with
// K.ellu, uniformly strided: then the address is arithmetic and the entry
// loads need not wait for the slice offset) entry k of slice row r is at
// 32 k + r; in the chunk-major copy laid out for LPR lanes per row it is at
// (k / LPR * 32 + r) * LPR + k % LPR (LPR 2 to 16).
template <int LPR>
__device__ __forceinline__ Row row_of_c(const DevEll& K, int row, int lr) {
  const int slice = row / kSliceH, rl = row - slice * kSliceH;
  Row r;
  if (LPR >= 2 && LPR <= 16 && K.cchunk == LPR) {
    r.e = K.ellc + (size_t)slice * K.cstride + (size_t)rl * LPR + lr;
  } else {
    const int2* base = K.ellu ? K.ellu + (size_t)slice * K.wu * kSliceH
                              : K.ell + __ldg(K.slice_off + slice);
    r.e = base + rl + (size_t)lr * kSliceH;
  }
  r.w = __ldg(K.slice_w + slice);
  return r;
}

// Lane lr's entry of the chunk starting at entry k0 (a multiple of LPR);
// padding {row, 0} past the slice width.
__device__ __forceinline__ int2 entry_at(const Row& r, int k0, int lr, int row) {
  if (k0 + lr >= r.w) return make_int2(row, 0);
  return r.na ? ldg_stream2(r.e + (size_t)k0 * kSliceH) : __ldg(r.e + (size_t)k0 * kSliceH);
}

// The entries of a row are read LPR at a time: each of the row's LPR lanes
// loads one entry of the chunk and the lanes hand them to each other with
// shuffles, so one load round trip serves LPR entries, and the next chunk is
// in flight while the gathers of the current one are issued.  `mask` holds
// every lane that takes part; w is the same for all rows of a warp (they
// share a slice), so the loops below are warp-uniform.  The neighbour loop
// is not unrolled: measured on GB300 against unroll 2 and 4 (and against a
// broadcast load of every entry), the lower register count wins overall
// (2D adjoint and tangent, 3D forward) and costs the 2D forward ~2%.
//
// MG_FOR_ENTRIES(LPR, r, row, lr, mask, cur, COL, V, BODY...) runs BODY with
// COL, V bound to entries 1 .. w-1 in order; `cur` must hold entry lr of the
// first chunk (entry_at(r, 0, lr, row)) on entry.
#define MG_FOR_ENTRIES(LPR, r, row, lr, mask, cur, COL, V, ...)                     \
  for (int k0_ = 0; k0_ < (r).w; k0_ += (LPR)) {                                    \
    const int2 nxt_ = entry_at((r), k0_ + (LPR), (lr), (row));                     \
    const int kn_ = min((LPR), (r).w - k0_);                                        \
    _Pragma("unroll 1") for (int k_ = k0_ == 0 ? 1 : 0; k_ < kn_; ++k_) {           \
      const int COL = __shfl_sync((mask), (cur).x, k_, (LPR));                       \
      const float V = __int_as_float(__shfl_sync((mask), (cur).y, k_, (LPR)));       \
      __VA_ARGS__                                                                    \
    }                                                                                \
    (cur) = nxt_;                                                                    \
  }

// acc[j] = sum_k K_k x[col_k][lane's float4 j], self[j] = x[row][...].
template <int LPR, int NV>
__device__ __forceinline__ void row_sum(const Row& r, const float* __restrict__ xb, int row,
                                        int lr, unsigned mask, int ld, float4 (&self)[NV],
                                        float4 (&acc)[NV]) {
  int2 cur = entry_at(r, 0, lr, row);
  const float* xr = xb + (size_t)row * ld;
#pragma unroll
  for (int j = 0; j < NV; ++j) self[j] = __ldg(reinterpret_cast<const float4*>(xr + 4 * LPR * j));
  const float v0 = __int_as_float(__shfl_sync(mask, cur.y, 0, LPR));
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = scale4(v0, self[j]);
  MG_FOR_ENTRIES(LPR, r, row, lr, mask, cur, col, v, {
    const float* xc = xb + (size_t)col * ld;
    float4 x[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) x[j] = __ldg(reinterpret_cast<const float4*>(xc + 4 * LPR * j));
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = fma4(v, x[j], acc[j]);
  })
}

template <int LPR, int NV>
__device__ __forceinline__ void row_sum2(const Row& r, const float* __restrict__ pb,
                                         const float* __restrict__ qb, int row, int lr,
                                         unsigned mask, int ld, float4 (&ps)[NV],
                                         float4 (&qs)[NV], float4 (&pacc)[NV],
                                         float4 (&qacc)[NV]) {
  int2 cur = entry_at(r, 0, lr, row);
  const size_t ro = (size_t)row * ld;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    ps[j] = __ldg(reinterpret_cast<const float4*>(pb + ro + 4 * LPR * j));
    qs[j] = __ldg(reinterpret_cast<const float4*>(qb + ro + 4 * LPR * j));
  }
  const float v0 = __int_as_float(__shfl_sync(mask, cur.y, 0, LPR));
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    pacc[j] = scale4(v0, ps[j]);
    qacc[j] = scale4(v0, qs[j]);
  }
  MG_FOR_ENTRIES(LPR, r, row, lr, mask, cur, col, v, {
    const size_t o = (size_t)col * ld;
    float4 x[NV], y[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      x[j] = __ldg(reinterpret_cast<const float4*>(pb + o + 4 * LPR * j));
      y[j] = __ldg(reinterpret_cast<const float4*>(qb + o + 4 * LPR * j));
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      pacc[j] = fma4(v, x[j], pacc[j]);
      qacc[j] = fma4(v, y[j], qacc[j]);
    }
  })
}

// Wide lanes: lane lr of a row holds the 8 consecutive shots [8 lr, 8 lr + 8)
// of the row's tile (two float4 side by side) instead of two float4 4 LPR
// shots apart, so each gather is one 32-byte load (ld.global.v8.f32, sm_100
// and later): half the load instructions for the same bytes.
struct F8 {
  float4 a, b;
};
__device__ __forceinline__ F8 ldg8(const float* p) {
  F8 r;
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r.a.x), "=f"(r.a.y), "=f"(r.a.z), "=f"(r.a.w), "=f"(r.b.x), "=f"(r.b.y),
        "=f"(r.b.z), "=f"(r.b.w)
      : "l"(p));
  return r;
}
// Loaded where it stands (after the gathers), like ld_pinned.
__device__ __forceinline__ F8 ld8_pinned(const float* p) {
  F8 r;
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(r.a.x), "=f"(r.a.y), "=f"(r.a.z), "=f"(r.a.w), "=f"(r.b.x), "=f"(r.b.y),
                 "=f"(r.b.z), "=f"(r.b.w)
               : "l"(p)
               : "memory");
  return r;
}
__device__ __forceinline__ void st8(float* p, const F8& v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v.a.x),
               "f"(v.a.y), "f"(v.a.z), "f"(v.a.w), "f"(v.b.x), "f"(v.b.y), "f"(v.b.z), "f"(v.b.w)
               : "memory");
}

// The row sum of row_sum with wide lanes (the same FMAs in the same order).
template <int LPR>
__device__ __forceinline__ void row_sum_w(const Row& r, const float* __restrict__ xb, int row,
                                          int lr, unsigned mask, int ld, F8& self, F8& acc) {
  int2 cur = entry_at(r, 0, lr, row);
  self = ldg8(xb + (size_t)row * ld);
  const float v0 = __int_as_float(__shfl_sync(mask, cur.y, 0, LPR));
  acc.a = scale4(v0, self.a);
  acc.b = scale4(v0, self.b);
  MG_FOR_ENTRIES(LPR, r, row, lr, mask, cur, col, v, {
    const F8 x = ldg8(xb + (size_t)col * ld);
    acc.a = fma4(v, x.a, acc.a);
    acc.b = fma4(v, x.b, acc.b);
  })
}
#undef MG_FOR_ENTRIES

// ---------------------------------------------------------------------------
// Pipelined gathers (kernels instantiated with R > 0).  The row sums above
// keep the NV float4 of one neighbour row in flight per lane: the next
// gather waits for the FMAs of the current one.  Here each lane copies the
// float4s it needs of the neighbour rows R - 1 entries ahead into its own
// slots of a shared-memory ring with 16-byte asynchronous copies (cp.async,
// cached in L1), one commit group per entry, and reads entry k back once
// its group has landed (cp.async.wait_group): R - 1 entries per lane are in
// flight and no register holds them.  A lane reads only what it copied
// itself, so no barrier is involved.  The entry's stiffness value is kept
// in the ring beside the data.  The arithmetic is that of the row sums
// above (the same FMAs in the same order), so the results carry the same
// bits.
//
// Ring of one CTA (dynamic shared memory): R slots per thread of NX float4
// (float4 j of slot s of thread t at (s * NX + j) * kThreads + t, so the 32
// lanes of a warp touch 512 contiguous bytes), then R floats per thread.
template <int NX, int R>
constexpr int ring_bytes() { return R == 0 ? 0 : kThreads * R * (16 * NX + 4); }

__device__ __forceinline__ void cp_async16(const void* smem, const float* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// acc[t][j] = sum_k K_k x_t[col_k][lane's float4 j], self[t][j] = x_t[row][...]
// for NS = 1 or 2 gathered states (x_1 unused when NS = 1).
template <int LPR, int NV, int NS, int R>
__device__ __forceinline__ void ring_sum(const Row& r, const float* __restrict__ x0,
                                         const float* __restrict__ x1, int row, int lr,
                                         unsigned mask, int ld, float4 (&self)[NS][NV],
                                         float4 (&acc)[NS][NV]) {
  static_assert(R >= 2 && (R & (R - 1)) == 0, "ring depth: a power of two");
  constexpr int A = R - 1, NX = NS * NV;
  extern __shared__ float4 ring_smem[];
  float4* rd = ring_smem;
  float* rv = reinterpret_cast<float*>(ring_smem + (size_t)R * NX * kThreads);
  const int tid = threadIdx.x;
  const float* xs[2] = {x0, x1};
  int2 cur = entry_at(r, 0, lr, row);        // issue side: entries [ib, ib + LPR)
  int2 nxt = entry_at(r, LPR, lr, row);  // and the next chunk, in flight
  int ib = 0;
  const float v0 = __int_as_float(__shfl_sync(mask, cur.y, 0, LPR));
  const size_t ro = (size_t)row * ld;
#pragma unroll
  for (int t = 0; t < NS; ++t)
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      self[t][j] = __ldg(reinterpret_cast<const float4*>(xs[t] + ro + 4 * LPR * j));
      acc[t][j] = scale4(v0, self[t][j]);
    }
  // copies of entry i (1 <= i < w) into slot i % R, as one commit group
  // (an empty group past the end of the row keeps the count uniform)
  auto issue = [&](int i) {
    if (i < r.w) {
      if (i >= ib + LPR) {
        cur = nxt;
        ib += LPR;
        nxt = entry_at(r, ib + LPR, lr, row);
      }
      const int col = __shfl_sync(mask, cur.x, i - ib, LPR);
      const float v = __int_as_float(__shfl_sync(mask, cur.y, i - ib, LPR));
      const int s = i & (R - 1);
      const size_t o = (size_t)col * ld;
#pragma unroll
      for (int t = 0; t < NS; ++t)
#pragma unroll
        for (int j = 0; j < NV; ++j)
          cp_async16(rd + (size_t)(s * NX + t * NV + j) * kThreads + tid,
                     xs[t] + o + 4 * LPR * j);
      rv[s * kThreads + tid] = v;
    }
    cp_commit();
  };
#pragma unroll
  for (int i = 1; i <= A; ++i) issue(i);
#pragma unroll 1
  for (int k = 1; k < r.w; ++k) {
    cp_wait<A - 1>();   // groups of entries 1..k have landed
    issue(k + A);       // into the slot read for entry k - 1
    const int s = k & (R - 1);
    const float v = rv[s * kThreads + tid];
#pragma unroll
    for (int t = 0; t < NS; ++t)
#pragma unroll
      for (int j = 0; j < NV; ++j)
        acc[t][j] = fma4(v, rd[(size_t)(s * NX + t * NV + j) * kThreads + tid], acc[t][j]);
  }
}

// The row sum of one state by plain loads (R = 0) or through the ring.
template <int LPR, int NV, int R>
__device__ __forceinline__ void gather1(const Row& r, const float* __restrict__ xb, int row,
                                        int lr, unsigned mask, int ld, float4 (&self)[NV],
                                        float4 (&acc)[NV]) {
  if constexpr (R == 0) {
    row_sum<LPR, NV>(r, xb, row, lr, mask, ld, self, acc);
  } else {
    float4 s1[1][NV], a1[1][NV];
    ring_sum<LPR, NV, 1, R>(r, xb, nullptr, row, lr, mask, ld, s1, a1);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      self[j] = s1[0][j];
      acc[j] = a1[0][j];
    }
  }
}

// The row sums of two states (forward and tangent) over the same entries.
template <int LPR, int NV, int R>
__device__ __forceinline__ void gather2(const Row& r, const float* __restrict__ pb,
                                        const float* __restrict__ qb, int row, int lr,
                                        unsigned mask, int ld, float4 (&ps)[NV],
                                        float4 (&qs)[NV], float4 (&pacc)[NV],
                                        float4 (&qacc)[NV]) {
  if constexpr (R == 0) {
    row_sum2<LPR, NV>(r, pb, qb, row, lr, mask, ld, ps, qs, pacc, qacc);
  } else {
    float4 s2[2][NV], a2[2][NV];
    ring_sum<LPR, NV, 2, R>(r, pb, qb, row, lr, mask, ld, s2, a2);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      ps[j] = s2[0][j];
      qs[j] = s2[1][j];
      pacc[j] = a2[0][j];
      qacc[j] = a2[1][j];
    }
  }
}

// Shot `s` of the batch as (float4 index j, component d) of this lane, or
// j = -1 when another lane (or another source tile) owns it.
template <int LPR, int NV>
__device__ __forceinline__ int owner(int s, int tile0, int lr, int& d) {
  const int rel = s - tile0;
  if (rel < 0 || rel >= 4 * LPR * NV) return -1;
  const int within = rel % (4 * LPR);
  if (within / 4 != lr) return -1;
  d = within % 4;
  return rel / (4 * LPR);
}

template <int NV>
__device__ __forceinline__ void add_to(float4 (&v)[NV], int j, int d, float x) {
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i == j) add_comp(v[i], d, x);
}

template <int NV>
__device__ __forceinline__ float get_from(const float4 (&v)[NV], int j, int d) {
  float out = 0.0f;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i == j) out = get_comp(v[i], d);
  return out;
}

// MINB > 1 asks the compiler for at least MINB resident CTAs per SM (a
// register cap): more warps in flight for the HBM-bound case, at the price
// of a few spilled registers in the rare source/receiver epilogue.
// A load the compiler keeps where it is written (after the row's gathers
// in the late-load form below).
__device__ __forceinline__ float4 ld_pinned(const float* p) {
  float4 v;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

// Prefetch of the line holding p into L1 (level 1) or L2 (level 2): the
// late loads of a capped kernel then find their rows on chip without
// holding registers across the gathers.
__device__ __forceinline__ void prefetch_to(const void* p, int level) {
  if (level == 1)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
  else
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ float2 ld_pinned2(const float2* p) {
  float2 v;
  asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
  return v;
}

// The forward step of row block `blk` (kWarps * 32 / LPR consecutive rows).
// LATE: the row's p_{l-1} and coefficients are loaded after its gathers, so
// that they hold no registers across the gather loop (the register-capped
// kernel then needs no spill slots in it).
template <int LPR, int NV, int R, bool LATE = false>
__device__ __forceinline__ void step_rows_block(const StepArgs& a, int blk) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blk * kWarps + warp) * RPW + lane / LPR;
  const unsigned mask = __ballot_sync(0xffffffffu, row < a.K.n);
  if (row >= a.K.n) return;
  const int lr = lane % LPR;
  const int tile0 = a.col0 + blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  Row r = row_of_c<LPR>(a.K, row, lr);
  r.na = a.stream;
  grid_dep_sync();
  const size_t ro = (size_t)row * a.ld + base;
  float4 c, old[NV], self[NV], acc[NV];
  if constexpr (LATE) {
    if (a.prefetch) {
      const int lv = a.prefetch == 1 ? 1 : 2;
      prefetch_to(a.coef + row, lv);
#pragma unroll
      for (int j = 0; j < NV; ++j) prefetch_to(a.pm + ro + 4 * LPR * j, lv);
    }
  }
  if constexpr (!LATE) {
    c = ld_coef(a.coef + row, a.stream);
#pragma unroll
    for (int j = 0; j < NV; ++j)
      old[j] = ld_once<false>(a.pm + ro + 4 * LPR * j, a.hint, a.stream);
  }
  gather1<LPR, NV, R>(r, a.p + base, row, lr, mask, a.ld, self, acc);
  if constexpr (LATE) {
    c = ld_pinned(reinterpret_cast<const float*>(a.coef + row));
#pragma unroll
    for (int j = 0; j < NV; ++j)
      old[j] = a.hint || a.stream ? ld_once<false>(a.pm + ro + 4 * LPR * j, a.hint, a.stream)
                                  : ld_pinned(a.pm + ro + 4 * LPR * j);
  }
  float4 out[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = leap(c, self[j], old[j], acc[j]);
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  const int s0 = __ldg(a.ev.src_ptr + row), s1 = __ldg(a.ev.src_ptr + row + 1);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.ev.src_shot + q), tile0, lr, d);
      if (j >= 0) add_to<NV>(out, j, d, sv);
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) st4(a.pout + ro + 4 * LPR * j, out[j]);
  if (a.traces) {
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.ev.rec_shot + q), tile0, lr, d);
      if (j >= 0) a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = get_from<NV>(out, j, d);
    }
  }
}

// One row block per CTA, or (a.sweep > 1) a.sweep consecutive row blocks
// per CTA, swept in order: the neighbour rows a block shares with the next
// are then still in the SM's L1.
// Prefetch level 3 of a swept CTA: before advancing block `blk`, each
// thread prefetches into L2 what its row of block blk + 1 reads first: its
// p_l and p_{l-1} segments, its coefficients and (uniformly strided
// stiffness) its first two chunks of entries.  Addresses only: no load, no
// register held.
template <int LPR, int NV>
__device__ __forceinline__ void prefetch_next_block(const StepArgs& a, int blk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = ((blk + 1) * kWarps + warp) * (32 / LPR) + lane / LPR;
  if (row >= a.K.n) return;
  const int lr = lane % LPR;
  const size_t ro = (size_t)row * a.ld + a.col0 + blockIdx.y * 4 * LPR * NV + 4 * lr;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    prefetch_to(a.p + ro + 4 * LPR * j, 2);
    prefetch_to(a.pm + ro + 4 * LPR * j, 2);
  }
  if (lr == 0) prefetch_to(a.coef + row, 2);
  if (LPR >= 2 && LPR <= 16 && a.K.cchunk == LPR) {   // the first two chunks of the row's entries
    const int s = row / kSliceH;
    const int2* e = a.K.ellc + (size_t)s * a.K.cstride + (size_t)(row - s * kSliceH) * LPR + lr;
    prefetch_to(e, 2);
    if (a.K.cstride > (int64_t)kSliceH * LPR) prefetch_to(e + (size_t)kSliceH * LPR, 2);
  } else if (a.K.ellu) {
    const int s = row / kSliceH;
    const int2* e = a.K.ellu + (size_t)s * a.K.wu * kSliceH + (row - s * kSliceH);
    if (lr < a.K.wu) prefetch_to(e + (size_t)lr * kSliceH, 2);
    if (lr + LPR < a.K.wu) prefetch_to(e + (size_t)(lr + LPR) * kSliceH, 2);
  }
}

template <int LPR, int NV, int MINB, int R>
__global__ void __launch_bounds__(kThreads, MINB) k_step_rows(StepArgs a) {
  constexpr bool kLate = MINB > 1;   // the register-capped form loads late
  if (a.sweep <= 1) {
    step_rows_block<LPR, NV, R, kLate>(a, blockIdx.x);
    return;
  }
  constexpr int RPB = kWarps * 32 / LPR;
  const int nblk = (a.K.n + RPB - 1) / RPB;
  const int b0 = blockIdx.x * a.sweep, b1 = min(b0 + a.sweep, nblk);
  for (int b = b0; b < b1; ++b) {
    if constexpr (kLate)
      if (a.prefetch == 3 && b + 1 < b1) prefetch_next_block<LPR, NV>(a, b);
    step_rows_block<LPR, NV, R, kLate>(a, b);
  }
}

// Shot s of the batch in the wide layout: float4 j and component d of this
// lane, or -1 when another lane (or another source tile) owns it.
template <int LPR>
__device__ __forceinline__ int owner_w(int s, int tile0, int lr, int& d) {
  const int rel = s - tile0;
  if (rel < 0 || rel >= 8 * LPR || rel / 8 != lr) return -1;
  d = rel % 4;
  return (rel % 8) / 4;
}

// The capped forward step of row block `blk` with wide lanes (two float4
// of consecutive shots per lane): the arithmetic of step_rows_block with
// LATE, same results.  Plain loads only (no cache-policy variants).
template <int LPR>
__device__ __forceinline__ void step_rows_block_w(const StepArgs& a, int blk) {
  constexpr int RPW = 32 / LPR, TW = 8 * LPR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blk * kWarps + warp) * RPW + lane / LPR;
  const unsigned mask = __ballot_sync(0xffffffffu, row < a.K.n);
  if (row >= a.K.n) return;
  const int lr = lane % LPR;
  const int tile0 = a.col0 + blockIdx.y * TW;
  const int base = tile0 + 8 * lr;
  const Row r = row_of_c<LPR>(a.K, row, lr);
  grid_dep_sync();
  const size_t ro = (size_t)row * a.ld + base;
  if (a.prefetch & 3) {
    const int lv = (a.prefetch & 3) == 1 ? 1 : 2;
    prefetch_to(a.coef + row, lv);
    prefetch_to(a.pm + ro, lv);
  }
  F8 self, acc;
  row_sum_w<LPR>(r, a.p + base, row, lr, mask, a.ld, self, acc);
  const float4 c = ld_pinned(reinterpret_cast<const float*>(a.coef + row));
  const F8 old = ld8_pinned(a.pm + ro);
  float4 out[2] = {leap(c, self.a, old.a, acc.a), leap(c, self.b, old.b, acc.b)};
  const int l = a.step + (a.step_base ? *a.step_base : 0);
  const int s0 = __ldg(a.ev.src_ptr + row), s1 = __ldg(a.ev.src_ptr + row + 1);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      int d;
      const int j = owner_w<LPR>(__ldg(a.ev.src_shot + q), tile0, lr, d);
      if (j >= 0) add_to<2>(out, j, d, sv);
    }
  }
  st8(a.pout + ro, F8{out[0], out[1]});
  if (a.traces) {
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      int d;
      const int j = owner_w<LPR>(__ldg(a.ev.rec_shot + q), tile0, lr, d);
      if (j >= 0) a.traces[(size_t)__ldg(a.ev.rec_trace + q) * a.nt + l] = get_from<2>(out, j, d);
    }
  }
}

template <int LPR, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_step_rows_w(StepArgs a) {
  if (a.sweep <= 1) {
    step_rows_block_w<LPR>(a, blockIdx.x);
    return;
  }
  constexpr int RPB = kWarps * 32 / LPR;
  const int nblk = (a.K.n + RPB - 1) / RPB;
  const int b0 = blockIdx.x * a.sweep, b1 = min(b0 + a.sweep, nblk);
  for (int b = b0; b < b1; ++b) {
    if ((a.prefetch & 3) == 3 && b + 1 < b1) prefetch_next_block<LPR, 2>(a, b);
    step_rows_block_w<LPR>(a, b);
  }
}

// The forward + tangent step of row block `blk`.  LATE as in
// step_rows_block: the row's own states and coefficients are loaded after
// its gathers.
template <int LPR, int NV, int R, bool LATE = false>
__device__ __forceinline__ void tangent_rows_block(const TangentArgs& a, int blk) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blk * kWarps + warp) * RPW + lane / LPR;
  const unsigned mask = __ballot_sync(0xffffffffu, row < a.f.K.n);
  if (row >= a.f.K.n) return;
  const int lr = lane % LPR;
  const int tile0 = a.f.col0 + blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  const int ld = a.f.ld;
  Row r = row_of_c<LPR>(a.f.K, row, lr);
  r.na = a.f.stream;
  grid_dep_sync();
  const size_t ro = (size_t)row * ld + base;
  float4 c, pold[NV], qold[NV], ps[NV], qs[NV], pacc[NV], qacc[NV];
  float2 tc;
  if constexpr (LATE) {
    if (a.f.prefetch) {
      prefetch_to(a.f.coef + row, a.f.prefetch);
      prefetch_to(a.tcoef + row, a.f.prefetch);
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        prefetch_to(a.f.pm + ro + 4 * LPR * j, a.f.prefetch);
        prefetch_to(a.qm + ro + 4 * LPR * j, a.f.prefetch);
      }
    }
  }
  if constexpr (!LATE) {
    c = ld_coef(a.f.coef + row, a.f.stream);
    tc = ld_coef(a.tcoef + row, a.f.stream);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      pold[j] = ld_once<false>(a.f.pm + ro + 4 * LPR * j, a.f.hint, a.f.stream);
      qold[j] = ld_once<false>(a.qm + ro + 4 * LPR * j, 0, a.f.stream);
    }
  }
  gather2<LPR, NV, R>(r, a.f.p + base, a.q + base, row, lr, mask, ld, ps, qs, pacc, qacc);
  if constexpr (LATE) {
    c = ld_pinned(reinterpret_cast<const float*>(a.f.coef + row));
    tc = ld_pinned2(a.tcoef + row);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      pold[j] = a.f.hint || a.f.stream ? ld_once<false>(a.f.pm + ro + 4 * LPR * j, a.f.hint,
                                                        a.f.stream)
                                       : ld_pinned(a.f.pm + ro + 4 * LPR * j);
      qold[j] = a.f.stream ? ld_once<false>(a.qm + ro + 4 * LPR * j, 0, a.f.stream)
                           : ld_pinned(a.qm + ro + 4 * LPR * j);
    }
  }
  float4 pn[NV], qn[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) pn[j] = leap(c, ps[j], pold[j], pacc[j]);
  const int l = a.f.step + (a.f.step_base ? *a.f.step_base : 0);
  const int s0 = __ldg(a.f.ev.src_ptr + row), s1 = __ldg(a.f.ev.src_ptr + row + 1);
  if (s0 != s1) {
    const float sv = c.z * __ldg(a.f.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.f.ev.src_shot + q), tile0, lr, d);
      if (j >= 0) add_to<NV>(pn, j, d, sv);
    }
  }
  // dp+ = alpha dp - beta dp- - gamma K dp - cm (p+ - 2p + p-) - cd (p+ - p-)
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    qn[j] = tangent_fix(leap(c, qs[j], qold[j], qacc[j]), pn[j], ps[j], pold[j], tc);
    st4(a.f.pout + ro + 4 * LPR * j, pn[j]);
    st4(a.qm + ro + 4 * LPR * j, qn[j]);
  }
  const int r0 = __ldg(a.f.ev.rec_ptr + row), r1 = __ldg(a.f.ev.rec_ptr + row + 1);
  for (int q = r0; q < r1; ++q) {
    int d;
    const int j = owner<LPR, NV>(__ldg(a.f.ev.rec_shot + q), tile0, lr, d);
    if (j >= 0) {
      const size_t at = (size_t)__ldg(a.f.ev.rec_trace + q) * a.f.nt + l;
      a.dtraces[at] = get_from<NV>(qn, j, d);
      if (a.f.traces) a.f.traces[at] = get_from<NV>(pn, j, d);   // forward traces too
    }
  }
}

// MINB > 1: the register cap of k_step_rows, with the late loads.
template <int LPR, int NV, int MINB, int R>
__global__ void __launch_bounds__(kThreads, MINB) k_tangent_rows(TangentArgs a) {
  tangent_rows_block<LPR, NV, R, (MINB > 1)>(a, blockIdx.x);
}

// Tangent step when the forward states are kept: p_{l-1}, p_l, p_{l+1} of
// the row are read (the forward field is not recomputed, so only dp is
// gathered); the dp update and its correction are those of k_tangent_rows,
// with the same bits.
template <int LPR, int NV, int R>
__global__ void __launch_bounds__(kThreads) k_tangent_kept_rows(TangentArgs a) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blockIdx.x * kWarps + warp) * RPW + lane / LPR;
  const unsigned mask = __ballot_sync(0xffffffffu, row < a.f.K.n);
  if (row >= a.f.K.n) return;
  const int lr = lane % LPR;
  const int tile0 = a.f.col0 + blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  const int ld = a.f.ld;
  Row r = row_of_c<LPR>(a.f.K, row, lr);
  r.na = a.f.stream;
  grid_dep_sync();
  const float4 c = ld_coef(a.f.coef + row, a.f.stream);
  const float2 tc = ld_coef(a.tcoef + row, a.f.stream);
  const size_t ro = (size_t)row * ld + base;
  float4 pn[NV], ps[NV], pold[NV], qold[NV], qs[NV], qacc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    pn[j] = ld_once<true>(a.pk1 + ro + 4 * LPR * j, 0, a.f.stream);
    ps[j] = ld_once<true>(a.f.p + ro + 4 * LPR * j, 0, a.f.stream);
    pold[j] = ld_once<true>(a.f.pm + ro + 4 * LPR * j, a.f.hint, a.f.stream);
    qold[j] = ld_once<false>(a.qm + ro + 4 * LPR * j, 0, a.f.stream);
  }
  gather1<LPR, NV, R>(r, a.q + base, row, lr, mask, ld, qs, qacc);
  float4 qn[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    qn[j] = tangent_fix(leap(c, qs[j], qold[j], qacc[j]), pn[j], ps[j], pold[j], tc);
    st4(a.qm + ro + 4 * LPR * j, qn[j]);
  }
  const int l = a.f.step + (a.f.step_base ? *a.f.step_base : 0);
  const int r0 = __ldg(a.f.ev.rec_ptr + row), r1 = __ldg(a.f.ev.rec_ptr + row + 1);
  for (int q = r0; q < r1; ++q) {
    int d;
    const int j = owner<LPR, NV>(__ldg(a.f.ev.rec_shot + q), tile0, lr, d);
    if (j >= 0) a.dtraces[(size_t)__ldg(a.f.ev.rec_trace + q) * a.f.nt + l] = get_from<NV>(qn, j, d);
  }
}

// 4-byte asynchronous copy global -> shared (no register holds the value
// while it is in flight); the issuing thread waits with cp.async.wait_all.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

// One compensated (Kahan) addition on values held in registers.
__device__ __forceinline__ void kahan_step(float& s, float& c, float term) {
  const float y = term - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// The reverse step of row block `blk`.  LATE as in step_rows_block.
template <int LPR, int NV, int R, bool LATE = false>
__device__ __forceinline__ void adjoint_rows_block(const AdjointArgs& a, int blk) {
  constexpr int RPW = 32 / LPR, TW = 4 * LPR * NV;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = (blk * kWarps + warp) * RPW + lane / LPR;
  const bool valid = row < a.K.n;
  const unsigned mask = __ballot_sync(0xffffffffu, valid);
  const int lr = lane % LPR;
  const int tile0 = a.col0 + blockIdx.y * TW;
  const int base = tile0 + 4 * lr;
  float t1 = 0.0f, t2 = 0.0f;
  // the row's accumulators (one set per source tile, read and written by
  // this row's lane 0 only in this launch) are copied to shared memory
  // before the gathers and updated at the end
  __shared__ float acc_s[kWarps * 32][4];
  float* mine = acc_s[warp * RPW + lane / LPR];
  if (valid) {
    Row r = row_of_c<LPR>(a.K, row, lr);
    r.na = a.stream;
    grid_dep_sync();
    if (lr == 0) {
      const size_t gi = (size_t)(tile0 / TW) * a.K.n + row;
      cp_async4(mine + 0, a.G + gi);
      cp_async4(mine + 1, a.Gc + gi);
      cp_async4(mine + 2, a.H + gi);
      cp_async4(mine + 3, a.Hc + gi);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    const size_t ro = (size_t)row * a.ld + base;
    float4 c, old[NV], pk[NV], self[NV], acc[NV];
    if constexpr (LATE) {
      if (a.prefetch) {
        prefetch_to(a.coef + row, a.prefetch);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
          prefetch_to(a.mu1 + ro + 4 * LPR * j, a.prefetch);
          prefetch_to(a.pk + ro + 4 * LPR * j, a.prefetch);
        }
      }
    }
    if constexpr (!LATE) {
      c = ld_coef(a.coef + row, a.stream);
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        old[j] = ld_once<false>(a.mu1 + ro + 4 * LPR * j, 0, a.stream);  // mu_{k+1}
        pk[j] = ld_once<true>(a.pk + ro + 4 * LPR * j, a.hint, a.stream);
      }
    }
    gather1<LPR, NV, R>(r, a.mu + base, row, lr, mask, a.ld, self, acc);
    if constexpr (LATE) {
      c = ld_pinned(reinterpret_cast<const float*>(a.coef + row));
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        old[j] = a.stream ? ld_once<false>(a.mu1 + ro + 4 * LPR * j, 0, a.stream)
                          : ld_pinned(a.mu1 + ro + 4 * LPR * j);
        pk[j] = a.hint || a.stream ? ld_once<true>(a.pk + ro + 4 * LPR * j, a.hint, a.stream)
                                   : ld_pinned(a.pk + ro + 4 * LPR * j);
      }
    }
    float4 out[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = leap(c, self[j], old[j], acc[j]);
    const int k = a.k + (a.step_base ? *a.step_base : 0);
    const int r0 = __ldg(a.ev.rec_ptr + row), r1 = __ldg(a.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      int d;
      const int j = owner<LPR, NV>(__ldg(a.ev.rec_shot + q), tile0, lr, d);
      if (j >= 0)
        add_to<NV>(out, j, d, c.w * __ldg(a.w + (size_t)__ldg(a.ev.rec_trace + q) * a.nt + (k - 1)));
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      st4(a.mu1 + ro + 4 * LPR * j, out[j]);
      adj_terms(pk[j], out[j], self[j], old[j], t1, t2);
    }
  }
#pragma unroll
  for (int off = LPR / 2; off > 0; off >>= 1) {
    t1 += __shfl_xor_sync(0xffffffffu, t1, off);
    t2 += __shfl_xor_sync(0xffffffffu, t2, off);
  }
  if (valid && lr == 0) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    float g = mine[0], gc = mine[1], h = mine[2], hc = mine[3];
    kahan_step(g, gc, t1);
    kahan_step(h, hc, t2);
    const size_t gi = (size_t)(tile0 / TW) * a.K.n + row;
    a.G[gi] = g;
    a.Gc[gi] = gc;
    a.H[gi] = h;
    a.Hc[gi] = hc;
  }
}

// MINB > 1: a register cap (6 resident CTAs per SM), with the late loads.
template <int LPR, int NV, int MINB, int R>
__global__ void __launch_bounds__(kThreads, MINB) k_adjoint_rows(AdjointArgs a) {
  adjoint_rows_block<LPR, NV, R, (MINB > 1)>(a, blockIdx.x);
}

// Launch shape for `cols` shot columns (a multiple of 4: a power of two up
// to 128 or a multiple of 128) and up to `nv` float4 per lane: the largest
// NV whose source tile of 4 * NV * LPR shots divides `cols`.
struct Shape {
  int lpr, nv;
  dim3 grid;
};

Shape shape_of(int n, int cols, int nv) {
  Shape s;
  for (;; nv >>= 1) {
    s.nv = nv;
    s.lpr = cols / (4 * nv) >= 32 ? 32 : cols / (4 * nv);
    // LPR must be a power of two (lanes of a row inside a warp)
    if (nv == 1 || (s.lpr >= 1 && (s.lpr & (s.lpr - 1)) == 0 && cols % (4 * nv * s.lpr) == 0))
      break;
  }
  const int rows_per_block = kWarps * (32 / s.lpr);
  s.grid = dim3((n + rows_per_block - 1) / rows_per_block, cols / (4 * s.nv * s.lpr));
  return s;
}

// Column range of a launch: col0 a multiple of the source tile, cols a
// whole number of tiles within ld.
bool range_ok(const Shape& sh, int col0, int cols, int ld) {
  const int tw = 4 * sh.nv * sh.lpr;
  return sh.lpr >= 1 && col0 >= 0 && cols > 0 && col0 + cols <= ld && col0 % tw == 0 &&
         cols % tw == 0;
}

// Raises a kernel's dynamic shared memory limit to `smem` bytes, once per
// kernel and device.
inline cudaError_t raise_smem_limit(const void* kern, int smem) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kern, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) done.insert({kern, dev});
  return e;
}

// Launch of a row kernel, dependent on the previous kernel of the stream
// (programmatic stream serialisation) when `pdl` is set, with `smem` bytes
// of dynamic shared memory (the gather ring; above 48 KB the kernel's limit
// is raised once per kernel and device).
template <class A>
cudaError_t launch_ex(void (*kern)(A), dim3 grid, int pdl, int smem, cudaStream_t st,
                      const A& a) {
  if (smem > 48 * 1024) {
    const cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// Largest dynamic shared memory a ring launch may ask for (227 KB per CTA).
constexpr int kRingSmemMax = 227 * 1024;

// Instantiation switch over the launch shape: KERN<LPR, NV, R> (or
// KERN<LPR, NV, M, R>) with the ring of NS gathered states.
#define MG_ROWS_SWITCH(KERN, R, NS, PDL, ARGS)                                                                \
  switch (sh.lpr * 8 + sh.nv) {                                                                               \
    case 32 * 8 + 1: err = launch_ex(KERN<32, 1, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break; \
    case 32 * 8 + 2: err = launch_ex(KERN<32, 2, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break; \
    case 32 * 8 + 4: err = launch_ex(KERN<32, 4, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break; \
    case 16 * 8 + 1: err = launch_ex(KERN<16, 1, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break; \
    case 16 * 8 + 2: err = launch_ex(KERN<16, 2, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break; \
    case 16 * 8 + 4: err = launch_ex(KERN<16, 4, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break; \
    case 8 * 8 + 1: err = launch_ex(KERN<8, 1, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 8 * 8 + 2: err = launch_ex(KERN<8, 2, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 8 * 8 + 4: err = launch_ex(KERN<8, 4, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    case 4 * 8 + 1: err = launch_ex(KERN<4, 1, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 4 * 8 + 2: err = launch_ex(KERN<4, 2, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 4 * 8 + 4: err = launch_ex(KERN<4, 4, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    case 2 * 8 + 1: err = launch_ex(KERN<2, 1, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 2 * 8 + 2: err = launch_ex(KERN<2, 2, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 2 * 8 + 4: err = launch_ex(KERN<2, 4, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    case 1 * 8 + 1: err = launch_ex(KERN<1, 1, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 1 * 8 + 2: err = launch_ex(KERN<1, 2, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 1 * 8 + 4: err = launch_ex(KERN<1, 4, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    default: return MG_ERR_ARG;                                                                               \
  }

#define MG_ROWS_SWITCH_M(KERN, M, R, NS, PDL, ARGS)                                                              \
  switch (sh.lpr * 8 + sh.nv) {                                                                                  \
    case 32 * 8 + 1: err = launch_ex(KERN<32, 1, M, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break; \
    case 32 * 8 + 2: err = launch_ex(KERN<32, 2, M, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break; \
    case 32 * 8 + 4: err = launch_ex(KERN<32, 4, M, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break; \
    case 16 * 8 + 1: err = launch_ex(KERN<16, 1, M, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break; \
    case 16 * 8 + 2: err = launch_ex(KERN<16, 2, M, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break; \
    case 16 * 8 + 4: err = launch_ex(KERN<16, 4, M, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break; \
    case 8 * 8 + 1: err = launch_ex(KERN<8, 1, M, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 8 * 8 + 2: err = launch_ex(KERN<8, 2, M, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 8 * 8 + 4: err = launch_ex(KERN<8, 4, M, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    case 4 * 8 + 1: err = launch_ex(KERN<4, 1, M, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 4 * 8 + 2: err = launch_ex(KERN<4, 2, M, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 4 * 8 + 4: err = launch_ex(KERN<4, 4, M, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    case 2 * 8 + 1: err = launch_ex(KERN<2, 1, M, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 2 * 8 + 2: err = launch_ex(KERN<2, 2, M, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 2 * 8 + 4: err = launch_ex(KERN<2, 4, M, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    case 1 * 8 + 1: err = launch_ex(KERN<1, 1, M, R>, sh.grid, PDL, ring_bytes<NS * 1, R>(), st, ARGS); break;   \
    case 1 * 8 + 2: err = launch_ex(KERN<1, 2, M, R>, sh.grid, PDL, ring_bytes<NS * 2, R>(), st, ARGS); break;   \
    case 1 * 8 + 4: err = launch_ex(KERN<1, 4, M, R>, sh.grid, PDL, ring_bytes<NS * 4, R>(), st, ARGS); break;   \
    default: return MG_ERR_ARG;                                                                                  \
  }

}  // namespace
}  // namespace mg
