// Read-only view of a mesh handle's resident data, for entry points that
// live outside capi.cu.
#pragma once

#include <cstdint>

#include "../../include/mgwave.h"
#include "kernels.cuh"

namespace mg {

struct MeshView {
  int device;
  int bc;
  int64_t n;                 // rows
  int64_t m;                 // finest cells
  DevEll K;                  // sliced-ELL stiffness
  CoefArgs coef_base;        // incidence arrays for the coefficients (eps, dt, outputs unset)
  const double* row_abs;     // sum_j |K_ij| per row (device)
  const int32_t* perm_host;  // caller node -> row (host, [n])
  int64_t* launches;         // the handle's launch counter
  int batch;                 // gather batch of the untiled kernels
};

int mesh_view(mg_mesh* mesh, MeshView* out);

}  // namespace mg
