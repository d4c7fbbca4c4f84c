/*
 * mgwave.h - C ABI of the GB300 leapfrog wave-propagation library.
 *
 * The library advances the scalar wave equation (pde1) of Takala, Us and
 * Pursiainen, "Multigrid-based inversion for volumetric radar imaging"
 * (Sec. II-A/II-B, App. A), discretised with nodal P1 elements on a nested
 * simplex mesh, by the explicit leapfrog of Eqs. (leap-frog1)-(leap-frog2)
 * with the flux eliminated:
 *
 *   (M + dt/2 D) p_{l+1} = 2 M p_l - (M - dt/2 D) p_{l-1} - dt^2 (K p_l - s_l e_src)
 *
 * K  P1 stiffness, K_ij = sum_e |e| grad phi_i . grad phi_j (App. A: the
 *    product sum_k B^(k)T A^-1 B^(k));
 * M  lumped eps-mass, m_i = sum_{e contains i} eps_e |e| / (d+1)
 *    (App. A's C, lumped);
 * D  first-order absorbing boundary (du/dn = -sqrt(eps) du/dt), lumped:
 *    D_ii = sum_{boundary facets F contains i} sqrt(eps_{e(F)}) |F| / d.
 *    It replaces App. A's split-field PML.
 * s  wavelet samples s_l = s(l dt); p_0 = p_{-1} = 0.
 *
 * Sample l of the trace of receiver node r of a shot is p_{l+1}[r].
 *
 * The Jacobian is the exact derivative of the traces with respect to the
 * permittivity of the cells of a chosen coarse level of the nested mesh
 * (Sec. II-B: eps_r = sum_j c_j chi'_j; the partial derivatives dp_l/dc_j).
 * Its tangent form is the auxiliary system of Eqs. (aku_ankka),
 * (linearized1)-(linearized2); its transpose is the discrete adjoint.
 *
 * Conventions for every call:
 *  - returns MG_OK (0) or a negative MG_ERR_* code; mg_strerror() names it;
 *  - node and cell ids are the caller's; the internal reordering is hidden;
 *  - the caller owns every input and output buffer; the mesh handle owns
 *    the device copy of the mesh and all scratch (states, checkpoints);
 *  - array arguments marked "data" are DEVICE pointers unless the call's
 *    flags contain MG_HOST_PTRS, in which case they are host pointers and
 *    the call copies them in and out itself and returns after the results
 *    have reached the host.  Shot descriptions are always host memory;
 *  - without MG_HOST_PTRS, work is queued on `stream` (a cudaStream_t, or
 *    NULL for the legacy default stream) and the call may return before it
 *    completes; outputs are valid once the stream has reached that point;
 *  - a handle must not be used by two calls at the same time (the scratch
 *    is shared); distinct handles are independent;
 *  - the current CUDA device at create time is the handle's device.
 */
#ifndef MGWAVE_H
#define MGWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MG_OK                 0
#define MG_ERR_ARG           -1  /* invalid argument (null, range, shape)   */
#define MG_ERR_NESTING       -2  /* parent maps do not describe a nesting   */
#define MG_ERR_OOM           -3  /* device allocation failed                */
#define MG_ERR_CUDA          -4  /* CUDA runtime error (no device, launch)  */
#define MG_ERR_CFL           -5  /* dt above the stability bound           */
#define MG_ERR_TIMEOUT       -6  /* a bounded device wait ran out           */
#define MG_ERR_UNSUPPORTED   -7  /* valid but not supported combination     */

/* ---- boundary modes ---------------------------------------------------- */
#define MG_BC_ABC1       0  /* first-order absorbing boundary (default)     */
#define MG_BC_NEUMANN    1  /* natural boundary, D = 0                      */
#define MG_BC_DIRICHLET  2  /* boundary nodes held at 0                      */

/* ---- mesh_create flags ------------------------------------------------- */
#define MG_ORDER_RCM     0  /* reverse Cuthill-McKee row order (default)    */
#define MG_ORDER_MORTON  1  /* Z-order of node coordinates                  */
#define MG_ORDER_NONE    2  /* caller order                                 */

/* ---- per-call flags ---------------------------------------------------- */
#define MG_HOST_PTRS        0x01  /* data pointers are host memory          */
#define MG_SINGLE_SOURCE    0x02  /* run the plain one-shot-at-a-time path   */
#define MG_NO_GRAPH         0x04  /* plain launches, no CUDA graph           */
#define MG_PERSISTENT       0x08  /* mg_forward: several steps per cooperative
                                     launch (mg_mesh_set_persistent)          */
#define MG_ALLOW_CFL        0x10  /* do not reject dt above the CFL bound    */
#define MG_KEEP_CHECKPOINTS 0x20  /* mg_forward: keep (p_l, p_{l-1}) every
                                     ckpt_every steps in the handle for a
                                     later mg_jacobian_T_apply               */
#define MG_REUSE_CHECKPOINTS 0x40 /* mg_jacobian_T_apply: use the
                                     checkpoints of the last mg_forward on
                                     this handle (same eps, shots, wavelet,
                                     dt, nt) instead of re-running it        */
#define MG_KEEP_STATES      0x80  /* mg_forward: keep every state p_0..p_nt
                                     in the handle ((nt + 2) n S_pad FP32,
                                     HBM permitting); a later
                                     mg_jacobian_T_apply with
                                     MG_REUSE_CHECKPOINTS and ckpt_every = nt
                                     then runs no recompute, and
                                     mg_jacobian_apply with
                                     MG_REUSE_CHECKPOINTS reads the forward
                                     field instead of recomputing it         */

typedef struct mg_mesh mg_mesh;

/* A batch of shots (host memory).  Shot k places the point source of
 * Eq. (pde1) at node src[k] (nodal load int delta_p phi_i = 1, App. A's
 * f_i) and records receivers rec[rec_ptr[k] .. rec_ptr[k+1]-1].  Trace rows
 * are numbered in that order: row r of a trace array belongs to the shot k
 * with rec_ptr[k] <= r < rec_ptr[k+1]. */
typedef struct {
  int32_t n_shots;
  const int32_t* src;      /* [n_shots]                   */
  const int64_t* rec_ptr;  /* [n_shots + 1], rec_ptr[0]=0 */
  const int32_t* rec;      /* [rec_ptr[n_shots]]          */
} mg_shots;

typedef struct {
  int32_t dim;
  int32_t n_levels;
  int64_t n_nodes;
  int64_t n_cells;        /* finest level                          */
  int64_t n_bnd;
  int64_t nnz;            /* stiffness non-zeros                   */
  int64_t ell_entries;    /* sliced-ELL entries incl. padding      */
  int32_t slice_height;
  int32_t max_row_nnz;
  int64_t device_bytes;   /* device memory held by the handle now  */
} mg_mesh_info_t;

/* Build a mesh handle (Sec. II-B nested meshes, App. A assembly).
 *  dim            2 (triangles) or 3 (tetrahedra)
 *  n_levels       L+1 >= 1 levels, level L the finest
 *  coords         [n_nodes][dim] float64, finest-level nodes (host)
 *  cells          [n_cells][dim+1] int32, finest-level cells (host)
 *  cell_parent    n_levels-1 host arrays; cell_parent[l-1][c] is the cell
 *                 of level l-1 containing cell c of level l (the nesting /
 *                 prolongation map).  May be NULL when n_levels == 1.
 *  n_cells_per_level [n_levels], last entry == n_cells
 *  bnd            [n_bnd][dim] int32 boundary facets (host); each must be a
 *                 facet of exactly one cell
 *  bc_mode        MG_BC_*
 *  order          MG_ORDER_*
 * Errors: MG_ERR_ARG (shapes, ids out of range, degenerate cell, facet not
 * on a cell), MG_ERR_NESTING (parent id out of range, a coarse cell with no
 * child), MG_ERR_CUDA / MG_ERR_OOM (device).  Argument checks run before
 * any CUDA call. */
int mg_mesh_create(int dim, int n_levels, const double* coords, int64_t n_nodes,
                   const int32_t* cells, int64_t n_cells,
                   const int32_t* const* cell_parent,
                   const int64_t* n_cells_per_level, const int32_t* bnd,
                   int64_t n_bnd, int bc_mode, int order, mg_mesh** out);

void mg_mesh_destroy(mg_mesh* mesh);

int mg_mesh_get_info(const mg_mesh* mesh, mg_mesh_info_t* info);

/* Internal row of each caller node id ([n_nodes] int32, host). */
int mg_mesh_get_permutation(const mg_mesh* mesh, int32_t* perm);

/* Stability bound dt_cfl = 2 / sqrt(max_i sum_j |K_ij| / m_i) (Gershgorin
 * bound of the largest eigenvalue of M^-1 K) for the permittivity eps
 * (data, [n_cells] float64).  Synchronous. */
int mg_cfl_dt(mg_mesh* mesh, const double* eps, int flags, void* stream,
              double* dt_out);

/* Forward traces (App. A leapfrog).
 *  eps      data, [n_cells] float64, > 0
 *  shots    host, see mg_shots
 *  wavelet  data, [nt] float64 samples s(l dt)
 *  traces   data, [rec_ptr[n_shots]][nt] float32 output
 *  ckpt_every  checkpoint spacing when MG_KEEP_CHECKPOINTS is set (>0)
 * All shots advance together in one node-major FP32 state (sources in the
 * fast dimension); MG_SINGLE_SOURCE runs them one at a time instead;
 * MG_PERSISTENT runs several steps per cooperative launch
 * (mg_mesh_set_persistent).  Flags: MG_HOST_PTRS, MG_NO_GRAPH,
 * MG_ALLOW_CFL, MG_SINGLE_SOURCE, MG_PERSISTENT, MG_KEEP_CHECKPOINTS,
 * MG_KEEP_STATES; any other bit is MG_ERR_UNSUPPORTED. */
int mg_forward(mg_mesh* mesh, const double* eps, const mg_shots* shots,
               const double* wavelet, double dt, int nt, float* traces,
               int ckpt_every, void* stream, int flags);

/* Forward traces without any allocation (the paper has no counterpart; this
 * is a service for callers that cannot let a library allocate).  Callers
 * that hand the whole device to their own memory pool, that must not pay
 * the implicit synchronisation of cudaMalloc/cudaFree inside a
 * latency-critical loop, or that need the call's memory footprint fixed in
 * advance can use it instead of mg_forward.  It computes the same traces as
 * mg_forward (same step kernel, same arithmetic) for device pointers only.
 *
 * All scratch (node order, per-row source/receiver lists, coefficients,
 * FP32 wavelet, two state buffers) lives in one file-scope device array of
 * 64 MiB that every GPU loading the library holds until the process exits.
 * It calls no cudaMalloc, cudaFree, graph instantiation or other allocating
 * routine, on the device or the host.
 *  - Size limit: 8 * n_nodes * S_pad + 44 * n_nodes + 4 * nt + 16 * shots
 *    + 12 * receivers bytes, plus up to 255 bytes of alignment for each of
 *    its 14 parts (S_pad = shot count rounded up to a power of two >= 4, or
 *    to a multiple of 128 above 128), must fit in 64 MiB; larger work
 *    returns MG_ERR_ARG before anything runs.
 *  - The array is reserved on a device, and its device address looked up
 *    there (cudaGetSymbolAddress), by mg_mesh_create on that device (a call
 *    that allocates anyway): the 64 MiB are taken then, even if this entry
 *    point is never called, and the call itself reserves no memory.
 *  - Every call on a device shares the one array, which keeps the previous
 *    call's contents (the call clears what must start at zero).  Calls whose
 *    work overlaps on the GPU (other streams, other threads, other handles)
 *    race on it: serialise them.
 *  - flags: 0 or MG_ALLOW_CFL; anything else returns MG_ERR_UNSUPPORTED.
 *  - eps, wavelet, traces: device pointers as in mg_forward; shots: host. */
int mg_forward_noalloc(mg_mesh* mesh, const double* eps, const mg_shots* shots,
                       const double* wavelet, double dt, int nt, float* traces,
                       void* stream, int flags);

/* Tangent: jv = J v, the derivative of the traces in the direction
 * eps_fine = eps + t * v[anc_level(e)] (Eqs. (aku_ankka), (linearized1)-
 * (linearized2), exact for the lumped scheme).
 *  level  0..n_levels-1, the mesh level that carries v
 *  v      data, [cells of level] float64
 *  jv     data, [rec_ptr[n_shots]][nt] float32 output
 *  flags  as mg_forward; with MG_REUSE_CHECKPOINTS the forward field is read
 *         from the history kept by the last mg_forward (or
 *         mg_forward_jacobian_apply) with MG_KEEP_STATES on this handle (same
 *         eps, shots, wavelet, dt, nt) instead of being advanced alongside:
 *         same bits, one sparse product per row instead of two; MG_ERR_ARG
 *         when no such history is kept. */
int mg_jacobian_apply(mg_mesh* mesh, int level, const double* eps,
                      const mg_shots* shots, const double* wavelet, double dt,
                      int nt, const double* v, float* jv, void* stream,
                      int flags);

/* The forward traces and the tangent J v in one pass: the tangent steps
 * advance p and dp together (as mg_jacobian_apply does), so recording p's
 * traces as well gives mg_forward's traces at no extra step.  Same traces
 * and J v bits as mg_forward and mg_jacobian_apply.  With MG_KEEP_STATES the
 * pass writes every forward state into the handle's kept history (as
 * mg_forward with MG_KEEP_STATES does), so that a later mg_jacobian_T_apply
 * with MG_REUSE_CHECKPOINTS and ckpt_every = nt needs no forward at all.
 *   traces, jv  [rec_ptr[n_shots]][nt] FP32 outputs (device, or host with
 *               MG_HOST_PTRS); other arguments as mg_jacobian_apply.
 *   flags       MG_HOST_PTRS, MG_ALLOW_CFL, MG_NO_GRAPH, MG_KEEP_STATES, and
 *               MG_PERSISTENT with MG_KEEP_STATES (several steps per
 *               cooperative launch, as mg_forward's; ends with a stream
 *               synchronisation, MG_ERR_TIMEOUT if a barrier wait ran out);
 *               MG_KEEP_CHECKPOINTS, MG_REUSE_CHECKPOINTS and
 *               MG_SINGLE_SOURCE return MG_ERR_UNSUPPORTED.
 * Row kernels only (the tiled tangent kernel does not record p). */
int mg_forward_jacobian_apply(mg_mesh* mesh, int level, const double* eps,
                              const mg_shots* shots, const double* wavelet, double dt, int nt,
                              const double* v, float* traces, float* jv, void* stream,
                              int flags);

/* Transpose: g = J^T w, the gradient of sum_{r,l} w[r][l] y[r][l] with
 * respect to the permittivity of each cell of `level`, by the discrete
 * adjoint (reverse-time leapfrog) with checkpoints every ckpt_every steps
 * and recomputation in between.
 *  w  data, [rec_ptr[n_shots]][nt] float32 trace weights
 *  g  data, [cells of level] float64 output
 *  flags  MG_HOST_PTRS, MG_NO_GRAPH, MG_ALLOW_CFL, MG_REUSE_CHECKPOINTS;
 *         MG_PERSISTENT when the reused checkpoints are a kept history
 *         (ckpt_every = nt after MG_KEEP_STATES): the reverse steps run
 *         several per cooperative launch, as mg_forward's (ends with a
 *         stream synchronisation; MG_ERR_TIMEOUT if a barrier wait ran
 *         out), else MG_ERR_UNSUPPORTED. */
int mg_jacobian_T_apply(mg_mesh* mesh, int level, const double* eps,
                        const mg_shots* shots, const double* wavelet, double dt,
                        int nt, const float* w, double* g, int ckpt_every,
                        void* stream, int flags);

/* Uneven batches: n_inst independent problems, each with its own handle
 * (distinct handles, one device), permittivity, shot batch, wavelet and dt,
 * all with the same step count nt.  The instances are cut, in the given
 * order, into groups whose states fit half of L2 (two states per instance
 * for the forward, three for J^T); a group of several instances is
 * advanced by ONE kernel launch per leapfrog step over a work list of
 * (instance, row block, source tile) items, an instance alone (one too
 * large to share L2) by its own tuned single-instance path.  Instance i
 * computes what mg_forward / mg_jacobian_T_apply would compute for it
 * alone (to FP32 rounding: the kernels differ).
 *  meshes, eps, wavelets, traces, w, g: arrays of n_inst pointers (host
 *  arrays; the pointed-to data are device pointers, or host pointers with
 *  MG_HOST_PTRS); shots, dts, levels: host arrays of n_inst entries.
 *  flags: MG_HOST_PTRS and/or MG_ALLOW_CFL.
 * Errors: MG_ERR_ARG (repeated handle, null entry), MG_ERR_UNSUPPORTED
 * (handles on different devices, other flags), plus the per-instance errors
 * of mg_forward. */
int mg_forward_batch(int n_inst, mg_mesh* const* meshes, const double* const* eps,
                     const mg_shots* shots, const double* const* wavelets, const double* dts,
                     int nt, float* const* traces, void* stream, int flags);

int mg_jacobian_T_apply_batch(int n_inst, mg_mesh* const* meshes, const int* levels,
                              const double* const* eps, const mg_shots* shots,
                              const double* const* wavelets, const double* dts, int nt,
                              const float* const* w, double* const* g, int ckpt_every,
                              void* stream, int flags);

/* Per-kernel tuning.  kind: MG_KERNEL_FORWARD (forward and recompute steps),
 * MG_KERNEL_TANGENT, MG_KERNEL_ADJOINT; batch / tile_rows / src_tile as in
 * mg_mesh_set_tuning (which sets all three kinds at once). */
#define MG_KERNEL_FORWARD 0
#define MG_KERNEL_TANGENT 1
#define MG_KERNEL_ADJOINT 2
int mg_mesh_set_kernel_tuning(mg_mesh* mesh, int kind, int batch, int tile_rows, int src_tile);

/* Shot groups of a kernel kind (kind = -1: all kinds): the padded shot
 * columns are split into `groups` equal groups (1, 2, 4 or 8) and, inside
 * each CUDA-graph chunk of steps (forward, tangent) and each checkpoint
 * segment (recompute, reverse), every group advances through all the steps
 * before the next group starts.  The shots are independent, so the results
 * are the same; the states a step touches shrink by the group count, which
 * lets them stay in L2 across consecutive steps.  A count whose group width
 * is not a power of two >= 4 up to 128 or a multiple of 128 runs as one
 * group; steps outside graphs run ungrouped.  Default 1.  Drops the cached
 * graphs.  Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_shot_groups(mg_mesh* mesh, int kind, int groups);

/* Register cap of the forward row kernel: 0 (none, default) or 5 (at least
 * five resident 256-thread CTAs per SM; more warps in flight for
 * HBM-bound meshes, a few spilled registers).  Drops the cached graphs.
 * Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_min_blocks(mg_mesh* mesh, int min_blocks);

/* The same register cap for a kernel kind: MG_KERNEL_FORWARD (as
 * mg_mesh_set_min_blocks), MG_KERNEL_TANGENT (the lockstep and fused
 * forward + tangent row kernel) or MG_KERNEL_ADJOINT (the reverse row
 * kernel; 5 or 6 resident CTAs per SM).  The capped kernels load the row's
 * own states and coefficients after its gathers, so that nothing is held
 * across the gather loop and the cap needs fewer spill slots there.  Same
 * results.  Drops the cached graphs.  Errors: MG_ERR_ARG for other kinds or
 * values (6 for a kind other than the adjoint). */
int mg_mesh_set_kernel_min_blocks(mg_mesh* mesh, int kind, int min_blocks);

/* Gather ring of the row kernels of a kernel kind (kind = -1: all kinds):
 * depth 4 or 8 makes every lane copy the float4s it needs of the neighbour
 * rows depth - 1 stiffness entries ahead into its own slots of a
 * shared-memory ring (16-byte cp.async through L1, one commit group per
 * entry) and read each back once it has landed, so several gathers per
 * lane are in flight without holding registers; 0 (default) gathers with
 * plain loads, one neighbour at a time.  Same arithmetic in the same
 * order: same results.  A launch shape whose ring exceeds a CTA's shared
 * memory (two gathered states of 4 float4 per lane at depth 8) fails with
 * MG_ERR_UNSUPPORTED.  Applies to the row kernels only (not to tiles or
 * the bulk-copy forward); ring kernels run without the register cap of
 * mg_mesh_set_kernel_min_blocks (the ring keeps the gathered values in
 * shared memory, not registers).  Drops the cached graphs.  Errors:
 * MG_ERR_ARG for other values. */
int mg_mesh_set_gather_ring(mg_mesh* mesh, int kind, int depth);

/* Row sweep of the forward row kernel: blocks > 1 makes each CTA advance
 * `blocks` consecutive row blocks (256 threads' rows each) one after
 * another instead of one, with a grid that many times smaller, so that the
 * neighbour rows a block shares with the next are still in the SM's L1.
 * 0 or 1 (default): one row block per CTA.  Same arithmetic: same results.
 * Drops the cached graphs.  Errors: MG_ERR_ARG outside 0..65536. */
int mg_mesh_set_row_sweep(mg_mesh* mesh, int blocks);
/* The forward row sweep (>= 0), or MG_ERR_ARG for a null handle. */
int mg_mesh_get_row_sweep(const mg_mesh* mesh);

/* Prefetch of the late-loaded rows of the register-capped row kernels
 * (mg_mesh_set_kernel_min_blocks) of a kernel kind (kind = -1: all kinds):
 * level 1 (L1) or 2 (L2) makes each lane prefetch the lines of its row's
 * own states and coefficients (p_{l-1}, and dp_{l-1} for the tangent;
 * mu_{k+1} and p_k for the adjoint) before the gathers, so the loads after
 * the gathers find them on chip without holding registers across the
 * gather loop; 0: none.  Uncapped kernels are not affected.  Same results.
 * Drops the cached graphs.  Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_late_prefetch(mg_mesh* mesh, int kind, int level);

/* Wide lanes of the register-capped forward row kernel with two float4 per
 * lane (on = 1): each lane holds 8 consecutive shots of its row, so that
 * every gather is one 32-byte load (sm_100 and later) instead of two
 * 16-byte loads.  Applies while mg_mesh_set_min_blocks(5) holds, the launch
 * shape has two float4 per lane, no L2 cache hint or L1 streaming applies
 * and the shot stride is a multiple of 8; otherwise the two-load kernel
 * runs.  Same arithmetic in the same order: same results.  Default 1
 * (measured faster: ellipsoid_3d forward 469.5 -> 463.4 us per step,
 * asteroid_2d 18.68 -> 18.52); 0: two 16-byte loads per gather.  Drops the
 * cached graphs.  Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_wide_lanes(mg_mesh* mesh, int on);

/* The switch above (0 or 1), or MG_ERR_ARG for a NULL handle. */
int mg_mesh_get_wide_lanes(const mg_mesh* mesh);

/* Chunk-major copy of the stiffness entries for the wide-lane forward with
 * `chunk` lanes per row (2, 4, 8 or 16; 0: off): entry k of row r of
 * slice s at s * stride + ((k / chunk) * 32 + r) * chunk + k % chunk, so a
 * warp's load of one chunk of entries for its rows reads consecutive
 * entries instead of one 32-entry column per lane.  Built on the device
 * from the handle's entries (host time and ceil(w_max / chunk) * 32 * chunk
 * * 8 bytes per slice of device memory); used by the wide-lane forward when
 * its launch shape has `chunk` lanes per row, ignored otherwise.  Same
 * results.  Drops the cached graphs.  Errors: MG_ERR_ARG for other values,
 * MG_ERR_OOM, MG_ERR_CUDA. */
int mg_mesh_set_chunked_ell(mg_mesh* mesh, int chunk);

/* The prefetch levels of the forward, tangent and adjoint kinds into
 * out[3].  Errors: MG_ERR_ARG for NULL arguments. */
int mg_mesh_get_late_prefetch(const mg_mesh* mesh, int32_t* out);

/* L1 policy of the row kernels of a kernel kind (kind = -1: all kinds):
 * 1 loads the data a step reads once (the row's own state values that are
 * not gathered, its coefficients and its stiffness entries) with
 * L1::no_allocate, so that L1 keeps the neighbour rows the gathers reuse;
 * 0 (default) loads them normally.  Same results.  Measured slower on
 * GB300 (three alternating runs on one box: ellipsoid_3d forward 535 ->
 * 556 us per step, the uneven batch's forward 842 -> 910 ms, the asteroid_2d
 * tangent and reverse steps 5-9%), so it stays off.  Drops the cached
 * graphs.  Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_l1_streaming(mg_mesh* mesh, int kind, int on);
/* That switch of the forward, tangent and adjoint kinds into out[3]. */
int mg_mesh_get_l1_streaming(const mg_mesh* mesh, int32_t* out);

/* Forward step on row tiles staged by the bulk-copy engine: rows > 0 (a
 * multiple of 32, at most 1024) makes the forward kind (forward, recompute
 * and kept-history steps) run a persistent kernel of one CTA per SM in
 * which a producer warp copies, per work item (a tile of `rows` Morton
 * rows and 32 shot columns), the tile's own and halo rows of p_l and its
 * local stiffness into one of two shared-memory buffers (cp.async.bulk on
 * mbarriers) while eight consumer warps compute the previous item from
 * shared memory.  Same arithmetic and bits as the row kernels.  Needs whole
 * 32-column items (padded shot counts of 32 or more) and a double buffer
 * that fits a CTA's shared memory, else the propagation call fails with
 * MG_ERR_UNSUPPORTED.  Its waits are bounded; a wait that runs out is
 * reported by mg_mesh_device_status.  0 (default) turns it off.  Measured
 * slower than the row kernels (ellipsoid_3d 2620 vs 538 us per step: the
 * copy engine takes the 128-byte row copies one at a time), so it is not
 * an autotuner candidate.  Drops the cached graphs.  Errors: MG_ERR_ARG for
 * other values. */
int mg_mesh_set_tma_tiles(mg_mesh* mesh, int rows);
/* Rows per tile of that kernel (0: off), or MG_ERR_ARG for a null handle. */
int mg_mesh_get_tma_tiles(const mg_mesh* mesh);

/* Generation of the handle's checkpoints and kept forward states: a count
 * (>= 0) that changes whenever a call writes, drops or invalidates them
 * (mg_forward, mg_forward_jacobian_apply, mg_jacobian_T_apply without
 * MG_REUSE_CHECKPOINTS, the batch calls, mg_mesh_trim, a conductivity
 * change).  A caller that keeps checkpoints for a later
 * mg_jacobian_T_apply with MG_REUSE_CHECKPOINTS records the generation
 * after its forward and asks for reuse only while it is unchanged: the
 * reuse check compares sizes, dt and shots, not the permittivity or the
 * wavelet.  MG_ERR_ARG for a null handle. */
int64_t mg_mesh_checkpoint_generation(const mg_mesh* mesh);

/* The multi-step forward (mg_forward with MG_PERSISTENT; App. A, Eqs.
 * (leap-frog1)-(leap-frog2), the same step as the single-step launches and
 * the same bits).  One cooperative launch advances `steps` leapfrog steps
 * (1..2^20, default 128; launches also end at every checkpoint): its CTAs,
 * all resident (at most the occupancy of the row kernel times the SM
 * count), sweep the row blocks of a step, then meet at a grid-wide barrier
 * before the next step.  A barrier wait is bounded by `wait_cycles` SM
 * clock cycles (>= 1000, default 2^31, about a second): a CTA that waits
 * longer, or that sees another CTA give up, records the time-out in the
 * handle's status word and leaves; mg_forward then synchronises with the
 * stream, clears the word and returns MG_ERR_TIMEOUT (its traces are
 * incomplete).  `extra_arrivals` (0..2^20; 0 in normal use) makes every
 * barrier wait for that many CTAs beyond the grid, which never arrive: it
 * exists to exercise the time-out path.  MG_PERSISTENT applies to
 * mg_forward only, without MG_SINGLE_SOURCE or MG_KEEP_STATES
 * (MG_ERR_UNSUPPORTED), uses the row kernel with the handle's float4 per
 * lane whatever the other tuning says, one shot group, no CUDA graph, and
 * ends with a stream synchronisation.  Errors: MG_ERR_ARG outside the
 * ranges above. */
int mg_mesh_set_persistent(mg_mesh* mesh, int steps, long long wait_cycles, int extra_arrivals);

/* Gather ring depth of the forward, tangent and adjoint kinds into out[3]. */
int mg_mesh_get_gather_ring(const mg_mesh* mesh, int32_t* out);

/* Forward step with the neighbour rows of each warp staged in shared
 * memory by bulk asynchronous copies (cp.async.bulk on an mbarrier) instead
 * of per-lane loads: same arithmetic and bits, more bytes in flight per
 * warp.  on: 0 (default) or 1.  Its waits are bounded; a wait that runs out
 * is reported by mg_mesh_device_status.  Drops the cached graphs. */
int mg_mesh_set_bulk_copies(mg_mesh* mesh, int on);

/* L2 cache policy of the kept-history path (MG_KEEP_STATES): 1 makes the
 * last read of each kept state in a pass (p_{l-1} in the forward and in the
 * tangent on kept states, p_k in the reverse steps) carry an evict-first
 * L2 policy, so that the lines still to be read stay in L2 while more
 * states stream than it holds.  Results are unchanged.  Default 1
 * (measured on the 2D bench step: forward 48.6 -> 42.7 ms and reverse steps
 * 72.5 -> 68.1 ms per 2000 steps); 0 loads them with the default policy.
 * Drops the cached graphs.  Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_cache_hints(mg_mesh* mesh, int on);

/* Uniformly strided stiffness copy for the row kernels: 1 builds (once) a
 * copy of the sliced ELL with every slice padded to the widest slice's
 * column count (padding {row, 0}), so a row's first entry address is
 * arithmetic and its entry loads need not wait for the slice offset.  Same
 * entries in the same order: same results.  Refused with
 * MG_ERR_UNSUPPORTED when the padding would more than double the stored
 * entries (meshes with very uneven row lengths).  0 returns to the sliced
 * layout.  Drops the cached graphs.  Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_uniform_ell(mg_mesh* mesh, int on);

/* Programmatic dependent launch of the row kernels (forward, tangent,
 * adjoint): 1 launches each step as a dependent of the previous kernel on
 * the stream, so that its CTAs are scheduled while the previous step's last
 * CTAs finish; every CTA reads the stiffness slice table, then waits for the
 * previous kernel to complete (griddepcontrol.wait) before touching any
 * state.  The arithmetic is unchanged: results are bit-identical.  1 is the
 * default (measured ~1% faster on the 2D bench step, neutral in 3D); 0
 * launches them in plain stream order.  Drops the cached graphs.
 * Errors: MG_ERR_ARG for other values. */
int mg_mesh_set_dependent_launch(mg_mesh* mesh, int on);

/* Status of the handle's bounded device waits since the last call:
 * MG_OK, MG_ERR_TIMEOUT (a wait ran out; the step it belongs to is
 * incomplete), MG_ERR_ARG (a copy address failed its alignment check).
 * Synchronises with the device and clears the status. */
int mg_mesh_device_status(mg_mesh* mesh);

/* Current tuning into out[17]: chunk, then (batch, tile_rows, src_tile,
 * groups, min_blocks) for the forward, tangent and adjoint kinds, then the
 * forward's bulk-copy switch. */
int mg_mesh_get_tuning(const mg_mesh* mesh, int32_t* out);

/* Autotuner: times every candidate launch shape of each kernel kind on the
 * caller's problem (steps leapfrog steps of mg_forward, mg_jacobian_apply
 * and mg_jacobian_T_apply on `level`, device pointers; wavelet must hold at
 * least `steps` samples), keeps the fastest per kind on the handle and
 * returns it in chosen[17] (may be NULL).  Candidates: row kernels with 1,
 * 2 or 4 float4 per lane; tiles of 64, 128 or 256 rows with 16 or 32 shots
 * per pass; row kernels under the register cap of 5 resident CTAs per SM
 * (mg_mesh_set_kernel_min_blocks; 1, 2 and 4 vectors per lane) and of 6
 * for the adjoint (1 and 2 vectors); row
 * kernels with 1, 2 or 4 float4 per lane and a gather ring of 4 or 8 slots
 * (mg_mesh_set_gather_ring; the chosen depths are read with
 * mg_mesh_get_gather_ring); for the forward the row kernels with 1 vector
 * per lane, and with 2 and 4 under the register cap, sweeping 4 row blocks
 * per CTA (mg_mesh_get_row_sweep); then 2, 4 and 8 shot groups on the two
 * fastest of those.  The handle's L1 streaming, prefetch, wide-lane and
 * stiffness-layout switches stay as they are.  Each
 * candidate is timed as the best of three runs after the GPU has been
 * warmed up; shapes within 1% of the fastest count as equal (the earliest
 * listed wins) and shot groups must win by more than 1%.  The choice is cached on
 * the handle per padded shot count; a
 * later call with the same count only re-applies it.  Synchronous.
 * flags: 0 or MG_ALLOW_CFL. */
int mg_autotune(mg_mesh* mesh, const double* eps, const mg_shots* shots, const double* wavelet,
                double dt, int steps, int level, void* stream, int flags, int32_t* chosen);

/* Projected data (Sec. II, "Projected data"): the time inner products
 *   <a, b>_1 = int_0^T a b dt,   <a, b>_2 = (1/T) int_0^T t a b dt
 * of every trace pair, with sample l of a trace at t_l = (l + 1) dt (the
 * state p_{l+1}), T = nt dt and the right-endpoint rectangle rule
 * (sum_l dt a_l b_l, and (1/T) sum_l dt t_l a_l b_l).  y^(j)_i = <u_i, u_i>_j
 * gives the projected data of traces u, y0^(j)_i = <u_i, u0_i>_j their
 * projection on simulated traces u0; y^(2)/y^(1) is the relative integrated
 * travel time of a pulse.  Since the measured u does not depend on the
 * parameters, the projected Jacobian is d<u, u0>_j / dc = <u, J_c u0>_j:
 * mg_project(u, J v) applies it, and mg_jacobian_T_apply with the weights of
 * mg_projected_weights applies its transpose.
 *   a, b: [n_traces][nt] FP32 traces; y: [2][n_traces] FP64 out (row 0
 *   <a_i, b_i>_1, row 1 <a_i, b_i>_2), accumulated in FP64 from the FP32
 *   samples in an order fixed by nt alone.
 *   flags: 0 (device pointers, asynchronous on `stream`) or MG_HOST_PTRS
 *   (host pointers; the call copies in and out and returns when y is on the
 *   host).
 * n_traces = 0 does nothing and succeeds (the pointers may then be NULL).
 * Errors: MG_ERR_ARG (null pointer, n_traces < 0, nt < 1, dt <= 0),
 * MG_ERR_UNSUPPORTED (other flags), MG_ERR_OOM, MG_ERR_CUDA. */
int mg_project(const float* a, const float* b, int64_t n_traces, int nt, double dt, double* y,
               void* stream, int flags);

/* Trace weights of the projected Jacobian transpose: for a cotangent z
 * ([2][n_traces] FP64) of the projected data <u_i, .>_j, the weights
 *   w_i(t_l) = dt (z[0][i] + z[1][i] t_l / T) u_i(t_l)
 * satisfy <w, d> = sum_{i,j} z[j][i] <u_i, d_i>_j for every trace
 * perturbation d, so mg_jacobian_T_apply(..., w, ...) returns J_proj^T z.
 *   u: [n_traces][nt] FP32; w: [n_traces][nt] FP32 out (FP64 arithmetic,
 *   rounded once).  flags, errors: as mg_project. */
int mg_projected_weights(const float* u, const double* z, int64_t n_traces, int nt, double dt,
                         float* w, void* stream, int flags);

/* TV-regularised reconstruction (Sec. II: reconstruction procedure,
 * Eq. (tv_iteration) with the regularisation matrix (d_mat); coarse-to-fine
 * approach, steps (1)-(5) with Eqs. (tv_iteration_0), (tv_iteration_2);
 * compression of coefficients) on the exact Jacobian of the data at eps0.
 *
 * Solves, for the level-cell perturbation x of the permittivity (x0 = 0),
 *   x_{l+1} = (L^T L + alpha D^T G_l D)^{-1} L^T dy,   G_0 = I,
 *   G_l = diag(|D x_l|)^{-1} (entries below 1e-8 max |D x_l| raised to it),
 * where L is the Jacobian of the data (traces, or projected data) with
 * respect to the cell values and D has D_ij = -s_ij / s_max for cells
 * sharing boundary measure s_ij and D_ii = beta + sum_j s_ij / s_max.
 * Every linear system is solved matrix-free by conjugate gradients with
 * FP64 vectors and inner products; each CG iteration applies L and L^T once
 * (mg_jacobian_apply, mg_jacobian_T_apply on checkpoints written once by
 * mg_forward at the start).
 *
 * level_f < 0: the single-level iteration on the cells of level_c.
 * level_f > level_c: coarse-to-fine; every outer step updates the level_c
 * cells, then solves for a correction in the fine fluctuations of level_f
 * (basis: +1/-1 on adjacent children of a coarse cell along a breadth-first
 * spanning tree of the children's facet adjacency rooted at the child with
 * most sibling neighbours; in 2D the centre-corner pairs), restricted to
 * the fluctuations of the ceil(keep_frac n_c) coarse cells with the largest
 * |x_c| and regularised by D_level_f applied to the fluctuation.
 *   data_mode  MG_DATA_TRACES: dy is [n_traces][nt] FP32 (y - y0), u unused.
 *              MG_DATA_PROJECTED: dy is [2][n_traces] FP64 projected data
 *              (see mg_project) and u the [n_traces][nt] FP32 traces they
 *              are projected on.
 *   x_out      [cells of level_f] (or of level_c) FP64: the final x.
 *   history    optional host array [n_outer][4]: CG iterations and final
 *              relative residual of the coarse and of the fine solve.
 *   flags      MG_HOST_PTRS (eps0, wavelet, dy, u, x_out on the host),
 *              MG_ALLOW_CFL.  Synchronous.
 * Errors: MG_ERR_ARG (levels, params out of range, null pointers),
 * MG_ERR_NESTING (children of a coarse cell not facet-connected), plus
 * those of the Jacobian calls. */
#define MG_DATA_TRACES    0
#define MG_DATA_PROJECTED 1
typedef struct {
  double alpha;      /* regularisation weight, > 0 */
  double beta;       /* diagonal weight of D, >= 0 */
  int n_outer;       /* outer iterations, >= 1 */
  int n_cg;          /* conjugate-gradient iterations per solve (upper bound), >= 1 */
  double cg_rtol;    /* CG stops at ||r|| <= cg_rtol ||b|| */
  double keep_frac;  /* compression: fraction of coarse cells kept, (0, 1] (paper: 1/3) */
  int ckpt_every;    /* checkpoint spacing of the adjoint, >= 1 */
} mg_tv_params;
int mg_tv_reconstruct(mg_mesh* mesh, int level_c, int level_f, const double* eps0,
                      const mg_shots* shots, const double* wavelet, double dt, int nt,
                      int data_mode, const void* dy, const float* u,
                      const mg_tv_params* params, double* x_out, double* history,
                      void* stream, int flags);

/* The coarse-to-fine reconstruction over more than two nested levels
 * (Sec. II, coarse-to-fine approach, the recursion (tv_iteration_3)).
 *  levels    host array of n_levels >= 1 strictly increasing mesh levels
 *            l_0 < l_1 < ... ; l_0 carries the coarse update, each further
 *            level l_i a correction in the fluctuations of l_i inside the
 *            cells of l_{i-1} (same basis, regulariser and compression as
 *            mg_tv_reconstruct's fine step).  The correction of l_i fits the
 *            data left by the coarse update and by the corrections of
 *            l_1..l_{i-1} of the same outer step (the printed sum of the
 *            recursion, its index read as running over the coarser levels);
 *            compression ranks the cells of l_{i-1} by |x| of the
 *            reconstruction assembled so far.  With {level_c} or
 *            {level_c, level_f} this is mg_tv_reconstruct.
 *  x_out     [cells of the last listed level] FP64.
 *  history   optional host array [n_outer][2 n_levels]: CG iterations and
 *            final relative residual of each level's solve, coarse first.
 * Other arguments, flags and errors as mg_tv_reconstruct. */
int mg_tv_reconstruct_levels(mg_mesh* mesh, const int* levels, int n_levels,
                             const double* eps0, const mg_shots* shots, const double* wavelet,
                             double dt, int nt, int data_mode, const void* dy, const float* u,
                             const mg_tv_params* params, double* x_out, double* history,
                             void* stream, int flags);

/* The paper's approximate Jacobian (App. A.1-A.3: auxiliary system,
 * Green's functions by reciprocity, multigrid approach, Eq. (approx_2)).
 *
 * For shot s (source a_s, one receiver r_s) and level cell j:
 *   L'_j(s)[l] = (|T'_j| / (d+1)) sum_{i in corners(j)} phi_{s,i}[l],
 *   phi_{s,i} = H_{i,r_s} * z_{s,i},  z_{s,i}[l] = -(p_{l+1} - 2 p_l + p_{l-1})_i / dt^2,
 * where p is the forward field of shot s, H_{i,r} the impulse response at
 * node i of a unit source (s_0 = 1) at r, equal by the symmetry of the
 * scheme to the response at r of a source at i, and corners(j) the d+1
 * corner nodes of cell j (the descendant vertices used by exactly one
 * descendant; MG_ERR_NESTING if a cell has not exactly d+1, i.e. the
 * refinement is not regular).  The auxiliary sources of a coarse cell sit
 * on its corners with the lumped coarse mass; the boundary-damping term of
 * the exact tangent is not included (the paper's auxiliary source carries
 * dC/dc only).  The Green's functions come from an impulse run rather than
 * the regularised deconvolution of App. A.2 (the impulse run is exact).
 * Cost: two batched forward runs recording every corner node, and FP32 FFT
 * convolutions.
 *   shots      exactly one receiver per shot (MG_ERR_UNSUPPORTED otherwise).
 *   u          [n_shots][nt] FP32 traces the columns are projected on
 *              (required with Lp, else may be NULL).
 *   Lp         optional out [2][n_shots][cells of level] FP64:
 *              <u_s, L'_j(s)>_k of Sec. II (projected data), k = 1, 2.
 *   phi        optional out [n_shots][n_nodes][nt] FP32 node responses.
 *   nodes      optional out [n_nodes] caller ids of the corner nodes, in
 *              the order of phi; n_nodes (required) receives their count.
 *              With Lp and phi both NULL only the node list is returned.
 *   mem_budget device bytes for the per-chunk work buffers (0: 8 GiB);
 *              shots are processed in chunks that fit.
 *   flags      MG_HOST_PTRS (eps, wavelet, u, Lp, phi host), MG_ALLOW_CFL.
 *              Synchronous. */
int mg_approx_jacobian(mg_mesh* mesh, int level, const double* eps, const mg_shots* shots,
                       const double* wavelet, double dt, int nt, const float* u, double* Lp,
                       float* phi, int32_t* nodes, int64_t* n_nodes, size_t mem_budget,
                       void* stream, int flags);

/* Forward traces of the paper's first-order leapfrog with element flux
 * variables and the split-field perfectly matched layer (App. A, Eqs.
 * (system1)-(system2), (leap-frog1)-(leap-frog2)):
 *   q^(k)_{l+1/2} = q^(k)_{l-1/2} + dt A^-1 (B^(k) p_l - T^(k) q^(k)_{l-1/2})
 *   p_{l+1}       = p_l + dt C^-1 (f_l - R p_l - S p_l - sum_k B^(k)T q^(k)_{l+1/2})
 * with A_ii = |T_i|, B^(k)_ij = |T_i| dphi_j/dx_k, C, R (the handle's
 * conductivity, evaluated explicitly as printed) and S = xi-mass lumped,
 * T^(k) = zeta^(k) A, f_l = dt sum_{m <= l} s_m.  The outer boundary is
 * natural (the handle's boundary mode is not used); the layer absorbs.
 * Sample l of a trace is p_{l+1} at the receiver.  With no layer and no
 * conductivity the traces equal mg_forward's with the Neumann boundary.
 *   xi    [n_cells] FP64 >= 0 per finest cell (caller order), or NULL.
 *   zeta  [n_cells][dim] FP64 >= 0 per finest cell and direction, or NULL.
 *   traces, shots, wavelet, dt, nt, flags (MG_HOST_PTRS, MG_ALLOW_CFL,
 *   MG_NO_GRAPH) as mg_forward; dt is checked against the CFL bound of
 *   mg_cfl_dt (the explicit damping terms need dt zeta and dt (sigma + xi)/eps
 *   below 1 in addition, which the caller chooses).  Synchronous; one launch
 *   per flux and per node update, whole chunks of the handle's graph chunk
 *   length replayed as one CUDA graph each (recorded once per call; step
 *   index read from a device counter the graph advances) unless
 *   MG_NO_GRAPH; the same results either way.
 * Errors: MG_ERR_ARG (null, negative zeta, degenerate cell), MG_ERR_CFL,
 * MG_ERR_UNSUPPORTED (other flags), MG_ERR_OOM, MG_ERR_CUDA. */
int mg_forward_pml(mg_mesh* mesh, const double* eps, const mg_shots* shots, const double* wavelet,
                   double dt, int nt, const double* xi, const double* zeta, float* traces,
                   void* stream, int flags);

/* Jacobian of mg_forward_pml's traces with respect to the cell permittivity
 * (App. A; only the eps-mass C depends on it), restricted to a level like
 * mg_jacobian_apply: jv = J v with eps_fine = eps + t v[anc_level(e)].
 * In lockstep with the forward, the fluxes of dp follow the flux update and
 *   dp_{l+1} = dp_l + dt C^-1 (-(R+S) dp_l - sum_k B^(k)T dq^(k)_{l+1/2})
 *              - (dC / C)(p_{l+1} - p_l),
 * dC the lumped mass of the direction (exact for the discrete scheme).
 *   level, v, jv  as mg_jacobian_apply ([cells of level] FP64 in,
 *                 [rec_ptr[n_shots]][nt] FP32 out);
 *   xi, zeta, the other arguments and flags as mg_forward_pml.
 * Synchronous.  Errors as mg_forward_pml, and MG_ERR_ARG for the level. */
int mg_jacobian_apply_pml(mg_mesh* mesh, int level, const double* eps, const mg_shots* shots,
                          const double* wavelet, double dt, int nt, const double* xi,
                          const double* zeta, const double* v, float* jv, void* stream,
                          int flags);

/* Gradient g = J^T w of mg_forward_pml's traces (the adjoint of the flux
 * leapfrog, App. A), g_c = sum over the level cell's descendants e of
 * d/deps_e sum_{r,l} w[r,l] y[r,l].  The forward keeps (p, q) every
 * ckpt_every steps; each segment's p states are recomputed, then the
 * adjoint steps run backwards: with a the adjoint of p_{l+1} and
 * r = a dt / C, the flux adjoint Qt^(k) = Q^(k)/|e| becomes
 * (1 - dt zeta_k) Qt^(k) - sum_a dphi_a/dx_k r[v_a], p_l receives
 * a - (R+S) r + dt sum_k B^(k)T Qt^(k), and the C-sensitivity gathers
 * -a (p_{l+1} - p_l) / C (FP64), turned into cells by |e|/(d+1).
 *   w        [rec_ptr[n_shots]][nt] FP32 trace weights;
 *   g        [cells of level] FP64 out;
 *   ckpt_every  checkpoint spacing >= 1 (memory: ceil(nt / ckpt_every)
 *            copies of p and q, and ckpt_every + 1 copies of p).
 * Each segment's recomputed p states are written straight into their
 * slots of the segment buffer; a full segment (recompute and reverse
 * steps) replays as one CUDA graph, as do chunks of the reverse steps when
 * one segment holds the whole run (unless MG_NO_GRAPH).
 * Other arguments and flags as mg_jacobian_apply_pml.  Synchronous. */
int mg_jacobian_T_apply_pml(mg_mesh* mesh, int level, const double* eps,
                            const mg_shots* shots, const double* wavelet, double dt, int nt,
                            const double* xi, const double* zeta, const float* w, double* g,
                            int ckpt_every, void* stream, int flags);

/* Nested prolongation of level-cell values to the finest cells (Sec. II-B:
 * eps_r = sum_j c_j chi'_j): out[e] = base[e] + v[anc_level(e)] for every
 * finest cell e (base may be NULL for 0).  v: [cells of level], base, out:
 * [n_cells]; data pointers (float64). */
int mg_prolong(mg_mesh* mesh, int level, const double* v, const double* base, double* out,
               void* stream, int flags);

/* Conductivity of the mesh (the sigma du/dt term of Eq. (pde1); the mass
 * matrix R of App. A weighted by sigma), used by every later call on the
 * handle.  Lumped like the eps-mass (R_ii = sum_{e contains i} sigma_e
 * |e|/(d+1)) and centred in time with the boundary damping:
 *   (M + dt/2 (D + R)) p_{l+1} = 2 M p_l - (M - dt/2 (D + R)) p_{l-1} - dt^2 (K p_l - s_l e).
 * sigma is a fixed nuisance parameter (Sec. III): the Jacobians remain
 * derivatives with respect to eps.  sigma: [n_cells] FP64 >= 0 (finest cells,
 * caller order), device pointer or host pointer with MG_HOST_PTRS (checked
 * there: MG_ERR_ARG for a negative or non-finite value); NULL removes it
 * (the default: no conductivity).  Invalidates kept checkpoints. */
int mg_mesh_set_conductivity(mg_mesh* mesh, const double* sigma, void* stream, int flags);

/* Release the handle's scratch (states, checkpoints, graphs). */
int mg_mesh_trim(mg_mesh* mesh);

/* Launch-shape tuning of a handle (no effect on results):
 *  chunk      leapfrog steps captured per CUDA graph; an even number >= 2,
 *             or 0 for one plain launch per step.  Default 128.
 *  batch      untiled kernels: float4 vectors (4 shots each) carried per
 *             lane, 1, 2 or 4.  Default 1.  More vectors share each row's
 *             stiffness loads among more shots and keep more neighbour
 *             loads in flight per lane.
 *  tile_rows  rows per shared-memory tile (a multiple of 32, <= 8192), or 0
 *             for the untiled kernels.  Default 0.  A tile stages its rows
 *             and their off-tile neighbours once per step and source tile.
 *  src_tile   shots staged per pass of a tile: 4, 8, 16, 32 or 64 (capped
 *             by the padded shot count).  Default 32.
 * A kernel whose tiled shared-memory footprint exceeds the device limit
 * runs untiled.  Pass -1 to keep a value.  Drops the cached graphs.
 * Errors: MG_ERR_ARG for values outside these sets. */
int mg_mesh_set_tuning(mg_mesh* mesh, int chunk, int batch, int tile_rows, int src_tile);

/* Number of kernel launches the handle has issued so far (graph-launched
 * kernels counted per node).  Used to report launch counts. */
int64_t mg_launch_count(const mg_mesh* mesh);

const char* mg_strerror(int code);

/* Library version, e.g. 100 for 0.1.0. */
int mg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MGWAVE_H */
