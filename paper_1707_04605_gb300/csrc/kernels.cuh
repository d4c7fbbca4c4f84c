// Device kernels of the leapfrog wave path and their launch wrappers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mg {

// Sparse stiffness in sliced-ELL form (see mg_internal.h).
struct DevEll {
  const int2* ell;          // {col, float bits of K_ij}
  const int64_t* slice_off;
  const int32_t* slice_w;
  int32_t n;                // rows
  const int2* ellu = nullptr;  // row kernels: the same entries with every slice
  int32_t wu = 0;              // padded to wu columns (slice s at s * wu * 32)
  // wide-lane forward with `cchunk` lanes per row: the same entries chunk
  // by chunk, entry k of row rl of slice s at
  // s * cstride + ((k / cchunk) * 32 + rl) * cchunk + k % cchunk
  const int2* ellc = nullptr;
  int32_t cchunk = 0;
  int64_t cstride = 0;
};

// Per-row event lists built from a shot batch: sources and receivers.
struct DevEvents {
  const int32_t* src_ptr;   // [n+1]
  const int32_t* src_shot;  // shot index of each source at the row
  const int32_t* rec_ptr;   // [n+1]
  const int32_t* rec_shot;  // shot index of each receiver entry at the row
  const int32_t* rec_trace; // trace row of each receiver entry
};

// One forward step, all shots: pout <- alpha p - beta pm - gamma (K p - s_l e_src)
// (state [n][ld] FP32, ld = padded shot count), records traces[tr][l].
struct StepArgs {
  DevEll K;
  DevEvents ev;
  const float4* coef;       // {alpha, beta, gamma, 1/w} per row
  const float* p;           // p_l
  const float* pm;          // p_{l-1}
  float* pout;              // p_{l+1} (may alias pm: in-place update)
  int32_t ld;
  const float* wavelet;     // FP32 samples
  float* traces;            // [n_traces][nt] or null
  int32_t nt;
  int32_t step;             // l = step + (step_base ? *step_base : 0)
  const int32_t* step_base;
  int32_t batch;            // row kernels: float4 vectors (4 shots each) per lane, 1/2/4
  int32_t min_blocks = 0;   // row kernel: 0, or 5 resident CTAs per SM requested (register cap)
  int32_t col0 = 0;         // first shot column advanced (multiple of the launch's shot tile)
  int32_t cols = 0;         // shot columns advanced, [col0, col0 + cols); 0 = all ld
  int32_t pdl = 0;          // row kernels: launch dependent on the previous kernel
  int32_t hint = 0;         // row kernels: L2 evict-first on the last read of pm
  int32_t ring = 0;         // row kernels: gather ring of 4 or 8 slots per lane (0 = plain loads)
  int32_t sweep = 0;        // forward row kernel: consecutive row blocks per CTA (0, 1: one)
  int32_t stream = 0;       // row kernels: once-read data loaded without L1 allocation
  int32_t prefetch = 0;     // capped row kernels: prefetch of the late-loaded rows (0, 1 L1, 2 L2)
  int32_t wide = 0;         // capped forward, two float4 per lane: 8 consecutive shots per lane
};

// Tangent step: forward and tangent states advance together.
struct TangentArgs {
  StepArgs f;               // forward (f.traces: forward traces, row kernel only, or null)
  const float* q;           // dp_l
  float* qm;                // dp_{l-1} in, dp_{l+1} out
  const float2* tcoef;      // {gamma dm/dt^2, gamma dD/(2 dt)} per row
  float* dtraces;           // [n_traces][nt]
  const float* pk1 = nullptr;  // kept p_{l+1}: f.p, f.pm, pk1 are kept forward states
                               // (read, not recomputed; f.pout unused)
};

// Adjoint (reverse) step k: mu_{k+1} buffer <- mu_{k-1}, and the per-row
// accumulations G += sum_s p_k (mu_{k-1} - 2 mu_k + mu_{k+1}),
// H += sum_s p_k (mu_{k-1} - mu_{k+1}) with Kahan compensation.
struct AdjointArgs {
  DevEll K;
  DevEvents ev;
  const float4* coef;
  const float* mu;          // mu_k
  float* mu1;               // mu_{k+1} in, mu_{k-1} out
  const float* pk;          // forward state p_k
  int32_t ld;
  const float* w;           // [n_traces][nt] trace weights
  int32_t nt;
  int32_t k;                // reverse step index k + (step_base ? *step_base : 0)
  const int32_t* step_base;
  int32_t batch;
  int32_t col0 = 0;         // shot columns [col0, col0 + cols) as in StepArgs
  int32_t cols = 0;
  int32_t pdl = 0;          // as in StepArgs
  int32_t hint = 0;         // row kernel: L2 evict-first on the read of pk
  int32_t ring = 0;         // row kernel: gather ring depth as in StepArgs
  int32_t stream = 0;       // row kernel: once-read loads without L1 allocation
  int32_t min_blocks = 0;   // row kernel: 0, or 5 or 6 resident CTAs per SM (register cap)
  int32_t prefetch = 0;     // as in StepArgs
  float* G;                 // [tiles][n] sums; row kernels: set = absolute source tile
  float* Gc;                // compensations
  float* H;
  float* Hc;
};

// Row tiles staged in shared memory (see HostTiles): tile t owns rows
// [t*P, t*P+P); its rows plus its halo rows are copied per source tile of
// `st_w` shots into shared memory and every neighbour read of the step is
// served from there through 16-bit local indices.
struct DevTiles {
  int32_t P;
  int32_t n_tiles;
  const int64_t* ell_off;
  const uint16_t* ell_idx;
  const float* ell_val;
  const int32_t* slice_info;  // {offset within tile, width} per global slice
  const int64_t* halo_off;
  const int32_t* halo_cnt;
  const int32_t* halo;
  int32_t max_ell;
  int32_t max_halo;
  int32_t st_w;               // shots per source tile (4..64, divides ld)
};

// Shared memory bytes of a tiled launch: kind 0 forward, 1 tangent, 2 adjoint.
size_t tiled_smem_bytes(const DevTiles& T, int kind);

int launch_step_tiled(const StepArgs& a, const DevTiles& T, cudaStream_t st);
int launch_tangent_tiled(const TangentArgs& a, const DevTiles& T, cudaStream_t st);
// Tangent step on kept forward states (row kernel; a.pk1 set).
int launch_tangent_kept(const TangentArgs& a, int S_pad, cudaStream_t st);
int launch_adjoint_tiled(const AdjointArgs& a, const DevTiles& T, cudaStream_t st);

// Source tiles (grid.y) of the row kernels for `cols` shot columns per
// launch and `nv` float4 per lane; the adjoint keeps one accumulator set per
// source tile of the whole padded shot range (S_pad / cols launches of
// rows_tiles(cols, nv) tiles each).
int rows_tiles(int cols, int nv);

int launch_step(const StepArgs& a, int S_pad, cudaStream_t st);
// Forward step with neighbour rows staged by bulk asynchronous copies
// (kernels_bulk.cu); err: device int set to 1 when a bounded wait ran out,
// 2 when a copy address was misaligned.
int launch_step_bulk(const StepArgs& a, int S_pad, int* err, cudaStream_t st);
// Forward step on row tiles staged by bulk copies with a producer warp and
// consumer warps (kernels_tma.cu); persistent grid of one CTA per SM, each
// sweeping a contiguous range of tiles in items of 32 shot columns.
// MG_ERR_UNSUPPORTED when the launch's columns are not whole 32-column
// items or its double buffer exceeds a CTA's shared memory; err: device int
// set to 1 when a bounded wait ran out.
int launch_step_tma(const StepArgs& a, const DevTiles& T, int S_pad, int* err, cudaStream_t st);
size_t tma_smem_bytes(const DevTiles& T);
int launch_step_single(const StepArgs& a, int shot, cudaStream_t st);
int launch_tangent(const TangentArgs& a, int S_pad, cudaStream_t st);
int launch_adjoint(const AdjointArgs& a, int S_pad, cudaStream_t st);
// Several forward steps in one cooperative launch (kernels_rows.cu): every
// CTA advances its row blocks (grid-stride) for step l, then all CTAs meet
// at a grid-wide barrier before step l + 1.  The barrier's wait is bounded:
// after `budget` SM clock cycles, or once another CTA has given up, a CTA
// sets *status = 1 and returns (the launch then ends without finishing its
// steps).  `extra` > 0 makes every barrier wait for arrivals that never
// come (tests of the time-out path); 0 otherwise.
struct PersistArgs {
  int32_t steps;            // leapfrog steps of the launch (a.step is the first)
  unsigned* count;          // barrier counter, zeroed by the launcher on the stream
  int* status;              // the handle's status word
  long long budget;         // SM clock cycles one barrier wait may take
  int32_t extra;            // arrivals awaited beyond the grid's CTAs
  float* seg = nullptr;     // kept history (tangent, adjoint): slot j holds p_{j-1}
  int64_t state = 0;        // floats per kept state
};
// a.pout must equal a.pm (in-place update).  MG_ERR_UNSUPPORTED when the
// device cannot hold the launch's source tiles as co-resident CTAs.
int launch_step_persist(const StepArgs& a, int S_pad, const PersistArgs& pa, cudaStream_t st);
// The fused forward + tangent step writing the kept history, pa.steps steps
// from a.f.step = l: p_l, p_{l-1}, p_{l+1} are slots l + 1, l, l + 2 of
// pa.seg; a.q / a.qm (dp_l, dp_{l-1}) swap roles after every step.
int launch_tangent_persist(const TangentArgs& a, int S_pad, const PersistArgs& pa,
                           cudaStream_t st);
// Reverse steps on the kept history, k = a.k, a.k - 1, ... (pa.steps of
// them): p_k is slot k + 1 of pa.seg; a.mu / a.mu1 swap roles after every
// step.
int launch_adjoint_persist(const AdjointArgs& a, int S_pad, const PersistArgs& pa,
                           cudaStream_t st);

// The same with the neighbour gathers pipelined through a shared-memory
// ring (kernels_ring.cu; called by the launchers above when ring > 0).
// MG_ERR_UNSUPPORTED when the ring of the launch shape exceeds a CTA's
// shared memory.
int launch_step_ring(const StepArgs& a, int S_pad, cudaStream_t st);
int launch_tangent_ring(const TangentArgs& a, int S_pad, cudaStream_t st);
int launch_tangent_kept_ring(const TangentArgs& a, int S_pad, cudaStream_t st);
int launch_adjoint_ring(const AdjointArgs& a, int S_pad, cudaStream_t st);

// Coefficients from eps (FP64 arithmetic, FP32 storage).
struct CoefArgs {
  int32_t n;
  const int64_t* nc_ptr; const int32_t* nc_cell; const double* nc_w;
  const int64_t* nf_ptr; const int32_t* nf_cell; const double* nf_w;
  const int32_t* is_bnd;
  const double* eps;
  double dt;
  int32_t bc;
  float4* coef;             // out
  double* mass;             // out (may be null)
  const double* sigma = nullptr;  // conductivity per finest cell, or null (none)
};
int launch_coefs(const CoefArgs& a, cudaStream_t st);

struct TangentCoefArgs {
  CoefArgs c;
  const double* v;          // level cells
  const int32_t* anc;       // ancestor on the level of each finest cell
  float2* tcoef;            // out
};
int launch_tangent_coefs(const TangentCoefArgs& a, cudaStream_t st);

// max_i row_abs_i / m_i -> out[0] (single block reduction).
int launch_cfl_reduce(int32_t n, const double* row_abs, const double* mass,
                      double* out, cudaStream_t st);

// g_e per finest cell from G, H; then restriction to level cells.
struct GradArgs {
  int64_t m;
  int32_t k;                // nodes per cell (d+1)
  int32_t dim;
  const int32_t* cells;     // [m][k] rows
  const double* vol;        // |e|
  const int64_t* cf_ptr;    // cell -> owned boundary facets
  const int32_t* cf_facet;
  const int32_t* bnd;       // [nb][dim] rows
  const double* bnd_meas;
  const double* eps;
  double dt;
  int32_t bc;
  int32_t n;
  int32_t tiles;
  const float* G; const float* Gc; const float* H; const float* Hc;
  double* g_fine;           // out [m]
};
int launch_cell_gradient(const GradArgs& a, cudaStream_t st);
int launch_restrict(int64_t nc, const int64_t* ptr, const int32_t* idx,
                    const double* g_fine, double* g_out, cudaStream_t st);

// out[e] = (base ? base[e] : 0) + v[anc[e]], e < m.
int launch_prolong(int64_t m, const int32_t* anc, const double* v, const double* base,
                   double* out, cudaStream_t st);

// Small helpers.
int launch_d2f(const double* in, float* out, int64_t n, cudaStream_t st);
int launch_add_int(int32_t* p, int32_t v, cudaStream_t st);
int launch_set_int(int32_t* p, int32_t v, cudaStream_t st);
int launch_copy_f4(const float* src, float* dst, int64_t n_floats, cudaStream_t st);

}  // namespace mg
