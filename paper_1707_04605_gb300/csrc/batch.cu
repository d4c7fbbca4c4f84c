// Uneven batches: several independent problems (own mesh handle, eps, shot
// batch, wavelet and dt; common step count).  The instances whose step
// alone is bound by launch latency are packed into groups whose states fit
// half of L2; each group of several instances is advanced by one kernel
// launch per leapfrog step over a work list of (instance, row block, source
// tile) items, so small instances share the GPU instead of leaving it idle,
// while every step still finds its states in L2; every other instance runs
// the tuned single-instance path.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <vector>

#include "../../include/mgwave.h"
#include "device_util.cuh"
#include "kernels.cuh"
#include "mesh_view.h"

namespace mg {
namespace {

using namespace dev;

struct Inst {
  DevEll K;
  DevEvents ev;
  const float4* coef;
  const float* wavelet;
  float* traces;     // [R][nt] or null
  float* A;          // forward: p_l lives in A for even l, in B for odd l
  float* B;
  float* seg;        // recompute: slot j holds p_{l0-1+j}
  float* mu;         // adjoint: mu_k lives in mu when nt-k is even
  float* mu1;
  const float* w;
  float* G;          // [4][tiles][n] Kahan accumulators
  int64_t state;     // n * ld
  int64_t acc;       // tiles * n
  int32_t ld, lpr;
};

struct Work {
  int32_t inst, row0, tile, pad;
};

constexpr int kBW = 8;  // warps per block

enum Mode { kForward = 0, kRecompute = 1 };

__device__ __forceinline__ float4 gather(const DevEll& K, int row, const float* __restrict__ p,
                                         int ld, int src0, float4& self) {
  const int slice = row / kSliceH;
  const int rl = row - slice * kSliceH;
  const int2* __restrict__ e = K.ell + __ldg(K.slice_off + slice) + rl;
  const int w = __ldg(K.slice_w + slice);
  self = __ldg(reinterpret_cast<const float4*>(p + (size_t)row * ld + src0));
  float4 acc = scale4(__int_as_float(__ldg(e).y), self);
#pragma unroll 4
  for (int k = 1; k < w; ++k) {
    const int2 ek = __ldg(e + k * kSliceH);
    acc = fma4(__int_as_float(ek.y),
               __ldg(reinterpret_cast<const float4*>(p + (size_t)ek.x * ld + src0)), acc);
  }
  return acc;
}

__global__ void __launch_bounds__(32 * kBW) k_step_multi(const Inst* __restrict__ insts,
                                                         const Work* __restrict__ work, int mode,
                                                         int l, int l0, int nt) {
  const Work wk = work[blockIdx.x];
  const Inst& I = insts[wk.inst];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lpr = I.lpr, rpw = 32 / lpr;
  const int row = wk.row0 + warp * rpw + lane / lpr;
  if (lane / lpr >= rpw || row >= I.K.n) return;
  const int src0 = wk.tile * 128 + (lane % lpr) * 4;
  const float *p, *pm;
  float* pout;
  if (mode == kForward) {
    p = (l & 1) ? I.B : I.A;
    pm = (l & 1) ? I.A : I.B;
    pout = const_cast<float*>(pm);
  } else {
    const int j = l - l0 + 1;
    p = I.seg + (size_t)j * I.state;
    pm = I.seg + (size_t)(j - 1) * I.state;
    pout = I.seg + (size_t)(j + 1) * I.state;
  }
  float4 self;
  const float4 acc = gather(I.K, row, p, I.ld, src0, self);
  const float4 c = __ldg(I.coef + row);
  const size_t ro = (size_t)row * I.ld + src0;
  const float4 old = *reinterpret_cast<const float4*>(pm + ro);
  float4 out = leap(c, self, old, acc);
  const int s0 = __ldg(I.ev.src_ptr + row), s1 = __ldg(I.ev.src_ptr + row + 1);
  if (s0 != s1) {
    const float sv = c.z * __ldg(I.wavelet + l);
    for (int q = s0; q < s1; ++q) {
      const int d = __ldg(I.ev.src_shot + q) - src0;
      if (d >= 0 && d < 4) add_comp(out, d, sv);
    }
  }
  st4(pout + ro, out);
  if (mode == kForward && I.traces) {
    const int r0 = __ldg(I.ev.rec_ptr + row), r1 = __ldg(I.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      const int d = __ldg(I.ev.rec_shot + q) - src0;
      if (d >= 0 && d < 4) I.traces[(size_t)__ldg(I.ev.rec_trace + q) * nt + l] = get_comp(out, d);
    }
  }
}

// 4-byte asynchronous copy global -> shared, waited for by the issuing
// thread (cp.async.wait_all): the row's accumulators are fetched while the
// step is computed instead of after it.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void kahan_step(float& s, float& c, float term) {
  const float y = term - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

__global__ void __launch_bounds__(32 * kBW) k_adjoint_multi(const Inst* __restrict__ insts,
                                                            const Work* __restrict__ work, int k,
                                                            int l0, int nt) {
  const Work wk = work[blockIdx.x];
  const Inst& I = insts[wk.inst];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lpr = I.lpr, rpw = 32 / lpr;
  const int row = wk.row0 + warp * rpw + lane / lpr;
  const bool valid = (lane / lpr < rpw) && row < I.K.n;
  const int src0 = wk.tile * 128 + (lane % lpr) * 4;
  const bool even = ((nt - k) & 1) == 0;
  const float* mu = even ? I.mu : I.mu1;
  float* mu1 = even ? I.mu1 : I.mu;
  float t1 = 0.0f, t2 = 0.0f;
  __shared__ float acc_s[kBW * 32][4];
  float* mine = acc_s[threadIdx.x];
  if (valid && (lane % lpr) == 0) {
    const size_t gi = (size_t)wk.tile * I.K.n + row;
    cp_async4(mine + 0, I.G + gi);
    cp_async4(mine + 1, I.G + I.acc + gi);
    cp_async4(mine + 2, I.G + 2 * I.acc + gi);
    cp_async4(mine + 3, I.G + 3 * I.acc + gi);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if (valid) {
    float4 self;
    const float4 acc = gather(I.K, row, mu, I.ld, src0, self);
    const float4 c = __ldg(I.coef + row);
    const size_t ro = (size_t)row * I.ld + src0;
    const float4 old = *reinterpret_cast<const float4*>(mu1 + ro);
    const float4 pk = __ldg(reinterpret_cast<const float4*>(I.seg + (size_t)(k - l0 + 1) * I.state + ro));
    float4 out = leap(c, self, old, acc);
    const int r0 = __ldg(I.ev.rec_ptr + row), r1 = __ldg(I.ev.rec_ptr + row + 1);
    for (int q = r0; q < r1; ++q) {
      const int d = __ldg(I.ev.rec_shot + q) - src0;
      if (d >= 0 && d < 4)
        add_comp(out, d, c.w * __ldg(I.w + (size_t)__ldg(I.ev.rec_trace + q) * nt + (k - 1)));
    }
    st4(mu1 + ro, out);
    adj_terms(pk, out, self, old, t1, t2);
  }
  // sum over the lanes of a row (lpr is a power of two, groups are aligned)
  for (int off = 16; off > 0; off >>= 1) {
    const float a1 = __shfl_xor_sync(0xffffffffu, t1, off);
    const float a2 = __shfl_xor_sync(0xffffffffu, t2, off);
    if (off < lpr) { t1 += a1; t2 += a2; }
  }
  if (valid && (lane % lpr) == 0) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    float g = mine[0], gc = mine[1], h = mine[2], hc = mine[3];
    kahan_step(g, gc, t1);
    kahan_step(h, hc, t2);
    const size_t gi = (size_t)wk.tile * I.K.n + row;
    I.G[gi] = g;
    I.G[I.acc + gi] = gc;
    I.G[2 * I.acc + gi] = h;
    I.G[3 * I.acc + gi] = hc;
  }
}

// Device copies of the instance table and the work list (grow-only).
struct Tables {
  std::mutex mu;
  void* p = nullptr;
  size_t bytes = 0;
  int dev = -1;
};
Tables g_tab;

int upload_tables(const std::vector<Inst>& insts, const std::vector<Work>& work, cudaStream_t st,
                  const Inst** di, const Work** dw) {
  const size_t bi = (insts.size() * sizeof(Inst) + 255) / 256 * 256;
  const size_t need = bi + work.size() * sizeof(Work);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MG_ERR_CUDA;
  if (g_tab.bytes < need || g_tab.dev != dev) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return MG_ERR_CUDA;
    if (g_tab.p && g_tab.dev == dev) cudaFree(g_tab.p);
    g_tab.p = nullptr;
    g_tab.bytes = 0;
    if (cudaMalloc(&g_tab.p, need) != cudaSuccess) { cudaGetLastError(); return MG_ERR_OOM; }
    g_tab.bytes = need;
    g_tab.dev = dev;
  }
  unsigned char* b = static_cast<unsigned char*>(g_tab.p);
  if (cudaMemcpyAsync(b, insts.data(), insts.size() * sizeof(Inst), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b + bi, work.data(), work.size() * sizeof(Work), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MG_ERR_CUDA;
  *di = reinterpret_cast<const Inst*>(b);
  *dw = reinterpret_cast<const Work*>(b + bi);
  return MG_OK;
}

void build_work(const std::vector<Inst>& insts, std::vector<Work>& work) {
  work.clear();
  for (int i = 0; i < (int)insts.size(); ++i) {
    const Inst& I = insts[i];
    const int rows = kBW * (32 / I.lpr);
    const int tiles = I.ld >= 128 ? I.ld / 128 : 1;
    for (int t = 0; t < tiles; ++t)
      for (int r = 0; r < I.K.n; r += rows) work.push_back({i, r, t, 0});
  }
}

Inst make_inst(const InstanceView& v, int nt) {
  Inst I{};
  I.K = v.K;
  I.ev = v.ev;
  I.coef = v.coef;
  I.wavelet = v.wavelet;
  I.A = v.A;
  I.B = v.B;
  I.seg = v.seg;
  I.mu = v.C;
  I.mu1 = v.D;
  I.w = v.w;
  I.G = v.G;
  I.state = v.n * v.S_pad;
  I.acc = (int64_t)v.tiles * v.n;
  I.ld = v.S_pad;
  I.lpr = v.S_pad >= 128 ? 32 : v.S_pad / 4;
  (void)nt;
  return I;
}

#define B_TRY(x) do { const int _rc = (x); if (_rc != MG_OK) return _rc; } while (0)
#define B_CU(x) do { if ((x) != cudaSuccess) { cudaGetLastError(); return MG_ERR_CUDA; } } while (0)

int check_batch(int n_inst, mg_mesh* const* meshes) {
  if (n_inst < 1 || !meshes) return MG_ERR_ARG;
  std::set<mg_mesh*> seen;
  int dev = -1;
  for (int i = 0; i < n_inst; ++i) {
    if (!meshes[i] || !seen.insert(meshes[i]).second) return MG_ERR_ARG;  // handles are distinct
    MeshView v;
    B_TRY(mesh_view(meshes[i], &v));
    if (dev >= 0 && v.device != dev) return MG_ERR_UNSUPPORTED;          // one device per batch
    dev = v.device;
  }
  return MG_OK;
}

// Node-shot updates per step below which one instance's step is bound by
// launch latency on its own: about 3.5 us per step of the single-instance
// path at ~400 G node-shot updates/s.
constexpr size_t kLatencyBoundWork = size_t(3) << 19;

// Grouping.  An instance with a step of at least kLatencyBoundWork updates
// runs alone on the tuned single-instance path (its autotuned kernels and
// CUDA graphs): a batched launch cannot do its work faster, and advancing
// it with others at every step would touch the states of all of them, which
// then stream from HBM once they exceed L2.  The latency-bound instances
// are packed, largest first, into groups whose working set (`states` padded
// states per instance) fits half of L2 (first fit), and each group of
// several runs the batched kernels.  Instances are independent, so the
// order in which groups run does not change any result.
std::vector<std::vector<int>> l2_groups(int n_inst, mg_mesh* const* meshes, const mg_shots* shots,
                                        int states) {
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0)
    l2 = 64 << 20;
  const size_t budget = (size_t)l2 / 2;
  std::vector<std::vector<int>> groups;
  std::vector<size_t> used;                 // working set of each packed group
  std::vector<std::pair<size_t, int>> small;   // (working set, instance)
  for (int i = 0; i < n_inst; ++i) {
    MeshView v;
    mesh_view(meshes[i], &v);
    const size_t cols = padded_shots(shots[i].n_shots);
    const size_t ws = (size_t)states * v.n * cols * sizeof(float);
    if ((size_t)v.n * cols >= kLatencyBoundWork || ws > budget)
      groups.push_back({i});
    else
      small.push_back({ws, i});
  }
  std::stable_sort(small.begin(), small.end(),
                   [](const std::pair<size_t, int>& x, const std::pair<size_t, int>& y) {
                     return x.first > y.first;
                   });
  const size_t first_packed = groups.size();
  for (const auto& [ws, i] : small) {
    size_t g = first_packed;
    while (g < groups.size() && used[g - first_packed] + ws > budget) ++g;
    if (g == groups.size()) {
      groups.push_back({});
      used.push_back(0);
    }
    groups[g].push_back(i);
    used[g - first_packed] += ws;
  }
  return groups;
}

// Forward of every instance over [0, nt); checkpoints (p_l, p_{l-1}) of
// instance i every ckpt_every steps when `views[i].ckpt` is set.
int run_batch_forward(std::vector<InstanceView>& views, std::vector<Inst>& insts, int nt,
                      int ckpt_every, cudaStream_t st, int64_t* launches) {
  for (auto& I : insts) {
    B_CU(cudaMemsetAsync(I.A, 0, I.state * sizeof(float), st));
    B_CU(cudaMemsetAsync(I.B, 0, I.state * sizeof(float), st));
  }
  std::vector<Work> work;
  build_work(insts, work);
  const Inst* di;
  const Work* dw;
  B_TRY(upload_tables(insts, work, st, &di, &dw));
  for (int l = 0; l < nt; ++l) {
    if (ckpt_every > 0 && l % ckpt_every == 0)
      for (size_t i = 0; i < insts.size(); ++i) {
        const Inst& I = insts[i];
        if (!views[i].ckpt) continue;
        float* slot = views[i].ckpt + (size_t)(l / ckpt_every) * 2 * I.state;
        const float* p = (l & 1) ? I.B : I.A;
        const float* pm = (l & 1) ? I.A : I.B;
        B_TRY(launch_copy_f4(p, slot, I.state, st));
        B_TRY(launch_copy_f4(pm, slot + I.state, I.state, st));
        *launches += 2;
      }
    k_step_multi<<<(unsigned)work.size(), 32 * kBW, 0, st>>>(di, dw, kForward, l, 0, nt);
    B_TRY(check_launch());
    *launches += 1;
  }
  return MG_OK;
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" int mg_forward_batch(int n_inst, mg_mesh* const* meshes, const double* const* eps,
                                const mg_shots* shots, const double* const* wavelets,
                                const double* dts, int nt, float* const* traces, void* stream,
                                int flags) {
  B_TRY(check_batch(n_inst, meshes));
  if (!eps || !shots || !wavelets || !dts || !traces || nt < 1) return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL)) return MG_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_inst; ++i)
    if (!traces[i]) return MG_ERR_ARG;
  for (const auto& grp : l2_groups(n_inst, meshes, shots, 2)) {
    if (grp.size() == 1) {
      const int i = grp[0];
      B_TRY(mg_forward(meshes[i], eps[i], &shots[i], wavelets[i], dts[i], nt, traces[i], 0, stream,
                       flags));
      continue;
    }
    const int n = (int)grp.size();
    std::vector<InstanceView> views(n);
    std::vector<Inst> insts(n);
    for (int j = 0; j < n; ++j) {
      const int i = grp[j];
      B_TRY(prepare_instance(meshes[i], eps[i], &shots[i], wavelets[i], dts[i], nt, flags, stream,
                             0, nullptr, &views[j]));
      insts[j] = make_inst(views[j], nt);
      insts[j].traces = views[j].tr;
    }
    B_TRY(run_batch_forward(views, insts, nt, 0, st, views[0].launches));
    for (int j = 0; j < n; ++j)
      B_CU(cudaMemcpyAsync(traces[grp[j]], views[j].tr, (size_t)views[j].R * nt * sizeof(float),
                           (flags & MG_HOST_PTRS) ? cudaMemcpyDeviceToHost
                                                  : cudaMemcpyDeviceToDevice,
                           st));
  }
  if (flags & MG_HOST_PTRS) B_CU(cudaStreamSynchronize(st));
  return MG_OK;
}

static int adjoint_group(int n_inst, mg_mesh* const* meshes, const int* levels,
                         const double* const* eps, const mg_shots* shots,
                         const double* const* wavelets, const double* dts, int nt,
                         const float* const* w, double* const* g, int ckpt_every, void* stream,
                         int flags);

extern "C" int mg_jacobian_T_apply_batch(int n_inst, mg_mesh* const* meshes, const int* levels,
                                         const double* const* eps, const mg_shots* shots,
                                         const double* const* wavelets, const double* dts, int nt,
                                         const float* const* w, double* const* g, int ckpt_every,
                                         void* stream, int flags) {
  B_TRY(check_batch(n_inst, meshes));
  if (!levels || !eps || !shots || !wavelets || !dts || !w || !g || nt < 1 || ckpt_every < 1)
    return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL)) return MG_ERR_UNSUPPORTED;
  for (int i = 0; i < n_inst; ++i)
    if (!w[i] || !g[i]) return MG_ERR_ARG;
  for (const auto& grp : l2_groups(n_inst, meshes, shots, 3)) {
    if (grp.size() == 1) {
      const int i = grp[0];
      B_TRY(mg_jacobian_T_apply(meshes[i], levels[i], eps[i], &shots[i], wavelets[i], dts[i], nt,
                                w[i], g[i], ckpt_every, stream, flags));
      continue;
    }
    std::vector<mg_mesh*> gm;
    std::vector<const double*> ge, gwv;
    std::vector<mg_shots> gs;
    std::vector<double> gdt;
    std::vector<int> gl;
    std::vector<const float*> gw;
    std::vector<double*> gg;
    for (int i : grp) {
      gm.push_back(meshes[i]); ge.push_back(eps[i]); gs.push_back(shots[i]);
      gwv.push_back(wavelets[i]); gdt.push_back(dts[i]); gl.push_back(levels[i]);
      gw.push_back(w[i]); gg.push_back(g[i]);
    }
    B_TRY(adjoint_group((int)grp.size(), gm.data(), gl.data(), ge.data(), gs.data(), gwv.data(),
                        gdt.data(), nt, gw.data(), gg.data(), ckpt_every, stream, flags));
  }
  return MG_OK;
}

// J^T w of one group of instances with the batched kernels.
static int adjoint_group(int n_inst, mg_mesh* const* meshes, const int* levels,
                  const double* const* eps, const mg_shots* shots,
                  const double* const* wavelets, const double* dts, int nt,
                  const float* const* w, double* const* g, int ckpt_every, void* stream,
                  int flags) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<InstanceView> views(n_inst);
  std::vector<Inst> insts(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    B_TRY(prepare_instance(meshes[i], eps[i], &shots[i], wavelets[i], dts[i], nt, flags, stream,
                           ckpt_every, w[i], &views[i]));
    insts[i] = make_inst(views[i], nt);
    insts[i].traces = nullptr;
  }
  int64_t* launches = views[0].launches;
  B_TRY(run_batch_forward(views, insts, nt, ckpt_every, st, launches));
  for (auto& I : insts) {
    B_CU(cudaMemsetAsync(I.mu, 0, I.state * sizeof(float), st));
    B_CU(cudaMemsetAsync(I.mu1, 0, I.state * sizeof(float), st));
    B_CU(cudaMemsetAsync(I.G, 0, 4 * I.acc * sizeof(float), st));
  }
  std::vector<Work> work;
  build_work(insts, work);
  const Inst* di;
  const Work* dw;
  B_TRY(upload_tables(insts, work, st, &di, &dw));
  const int nck = (nt + ckpt_every - 1) / ckpt_every;
  for (int a = nck - 1; a >= 0; --a) {
    const int l0 = a * ckpt_every;
    const int l1 = std::min(nt, l0 + ckpt_every);
    for (size_t i = 0; i < insts.size(); ++i) {
      const Inst& I = insts[i];
      B_TRY(launch_copy_f4(views[i].ckpt + (size_t)a * 2 * I.state, I.seg + I.state, I.state, st));
      B_TRY(launch_copy_f4(views[i].ckpt + (size_t)a * 2 * I.state + I.state, I.seg, I.state, st));
      *launches += 2;
    }
    for (int l = l0; l < l1; ++l) {
      k_step_multi<<<(unsigned)work.size(), 32 * kBW, 0, st>>>(di, dw, kRecompute, l, l0, nt);
      B_TRY(check_launch());
      *launches += 1;
    }
    for (int k = l1; k > l0; --k) {
      k_adjoint_multi<<<(unsigned)work.size(), 32 * kBW, 0, st>>>(di, dw, k, l0, nt);
      B_TRY(check_launch());
      *launches += 1;
    }
  }
  for (int i = 0; i < n_inst; ++i)
    B_TRY(finish_gradient(meshes[i], levels[i], views[i].eps, dts[i], views[i].tiles, g[i], flags,
                          stream));
  return MG_OK;
}
