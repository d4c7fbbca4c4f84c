// Launchers of the row kernels (rows_common.cuh) whose neighbour gathers
// are pipelined through a per-thread shared-memory ring of R = 4 or 8 slots
// (R - 1 entries in flight per lane; see ring_sum).  Same arithmetic and
// bits as the plain launches of kernels_rows.cu.
#include "rows_common.cuh"

namespace mg {
namespace {

// Ring depth R of a launch is 4 or 8, and its shared memory must fit a CTA.
int ring_check(int ring, int ns, int nv) {
  if (ring != 4 && ring != 8) return MG_ERR_ARG;
  const long bytes = (long)kThreads * ring * (16L * ns * nv + 4);
  return bytes <= kRingSmemMax ? MG_OK : MG_ERR_UNSUPPORTED;
}

}  // namespace

int launch_step_ring(const StepArgs& a, int S_pad, cudaStream_t st) {
  const int cols = a.cols ? a.cols : S_pad;
  Shape sh = shape_of(a.K.n, cols, a.batch);
  if (a.sweep > 1) sh.grid.x = (sh.grid.x + a.sweep - 1) / a.sweep;
  if (!range_ok(sh, a.col0, cols, a.ld)) return MG_ERR_ARG;
  if (int rc = ring_check(a.ring, 1, sh.nv)) return rc;
  cudaError_t err = cudaSuccess;
  if (a.ring == 4) {
    MG_ROWS_SWITCH_M(k_step_rows, 1, 4, 1, a.pdl, a)
  } else {
    MG_ROWS_SWITCH_M(k_step_rows, 1, 8, 1, a.pdl, a)
  }
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

int launch_tangent_ring(const TangentArgs& a, int S_pad, cudaStream_t st) {
  const int cols = a.f.cols ? a.f.cols : S_pad;
  const Shape sh = shape_of(a.f.K.n, cols, a.f.batch);
  if (!range_ok(sh, a.f.col0, cols, a.f.ld)) return MG_ERR_ARG;
  if (int rc = ring_check(a.f.ring, 2, sh.nv)) return rc;
  cudaError_t err = cudaSuccess;
  if (a.f.ring == 4) {
    MG_ROWS_SWITCH_M(k_tangent_rows, 1, 4, 2, a.f.pdl, a)
  } else {
    MG_ROWS_SWITCH_M(k_tangent_rows, 1, 8, 2, a.f.pdl, a)
  }
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

int launch_tangent_kept_ring(const TangentArgs& a, int S_pad, cudaStream_t st) {
  const int cols = a.f.cols ? a.f.cols : S_pad;
  const Shape sh = shape_of(a.f.K.n, cols, a.f.batch);
  if (!range_ok(sh, a.f.col0, cols, a.f.ld) || !a.pk1) return MG_ERR_ARG;
  if (int rc = ring_check(a.f.ring, 1, sh.nv)) return rc;
  cudaError_t err = cudaSuccess;
  if (a.f.ring == 4) {
    MG_ROWS_SWITCH(k_tangent_kept_rows, 4, 1, a.f.pdl, a)
  } else {
    MG_ROWS_SWITCH(k_tangent_kept_rows, 8, 1, a.f.pdl, a)
  }
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

int launch_adjoint_ring(const AdjointArgs& a, int S_pad, cudaStream_t st) {
  const int cols = a.cols ? a.cols : S_pad;
  const Shape sh = shape_of(a.K.n, cols, a.batch);
  if (!range_ok(sh, a.col0, cols, a.ld)) return MG_ERR_ARG;
  if (int rc = ring_check(a.ring, 1, sh.nv)) return rc;
  cudaError_t err = cudaSuccess;
  if (a.ring == 4) {
    MG_ROWS_SWITCH_M(k_adjoint_rows, 1, 4, 1, a.pdl, a)
  } else {
    MG_ROWS_SWITCH_M(k_adjoint_rows, 1, 8, 1, a.pdl, a)
  }
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

}  // namespace mg
