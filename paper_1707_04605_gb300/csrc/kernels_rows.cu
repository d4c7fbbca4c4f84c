// Launchers of the row kernels (rows_common.cuh) with plain neighbour
// gathers; a launch that asks for the gather ring (a.ring / a.f.ring > 0)
// goes to kernels_ring.cu.
#include "rows_common.cuh"

namespace mg {

int rows_tiles(int cols, int nv) { return (int)shape_of(1, cols, nv).grid.y; }

int launch_step(const StepArgs& a, int S_pad, cudaStream_t st) {
  if (a.ring) return launch_step_ring(a, S_pad, st);
  const int cols = a.cols ? a.cols : S_pad;
  Shape sh = shape_of(a.K.n, cols, a.batch);
  if (a.sweep > 1) sh.grid.x = (sh.grid.x + a.sweep - 1) / a.sweep;
  if (!range_ok(sh, a.col0, cols, a.ld)) return MG_ERR_ARG;
  cudaError_t err = cudaSuccess;
  if (a.min_blocks == 5) {
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
  MG_ROWS_SWITCH(k_tangent_rows, 0, 2, a.f.pdl, a)
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
  MG_ROWS_SWITCH(k_adjoint_rows, 0, 1, a.pdl, a)
  if (err != cudaSuccess) return MG_ERR_CUDA;
  return check_launch();
}

}  // namespace mg
