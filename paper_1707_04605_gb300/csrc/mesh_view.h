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

// Padded shot count (row stride of the states) of a batch of S shots.
int padded_shots(int S);

// Loads the module of mg_forward_noalloc's fixed device array and its
// kernels on device `dev` (current) and caches the array's address there.
int noalloc_prepare(int dev);

struct HostMesh;
// Host image of a handle's mesh (read-only), its device, and a way to count
// launches made on its behalf by entry points outside capi.cu.
const HostMesh* host_mesh(const mg_mesh* mesh);
int mesh_device(const mg_mesh* mesh);
int mesh_graph_chunk(const mg_mesh* mesh);   // steps per CUDA-graph chunk (0: off)
void add_launches(mg_mesh* mesh, int64_t n);

// One problem of a multi-instance batch, prepared on its own handle: device
// inputs staged, coefficients and FP32 wavelet computed, event lists built,
// and the handle's state / checkpoint / accumulator buffers sized.
struct InstanceView {
  DevEll K;
  DevEvents ev;
  const float4* coef;
  const float* wavelet;
  const double* eps;        // device copy or caller pointer
  int S, S_pad, tiles;
  int64_t R, n;
  float* A; float* B; float* C; float* D;  // n * S_pad floats each
  float* ckpt;              // [nck][2][n][S_pad] when requested
  float* seg;               // [K+2][n][S_pad] when requested
  float* tr;                // [R][nt] internal trace buffer
  float* G;                 // [4][tiles][n] Kahan accumulators when requested
  const float* w;           // [R][nt] staged weights when given
  int64_t* launches;
};

// ckpt_every > 0 sizes checkpoint and segment buffers; w (device or host
// per flags) is staged when non-null.
int prepare_instance(mg_mesh* mesh, const double* eps, const mg_shots* shots,
                     const double* wavelet, double dt, int nt, int flags, void* stream,
                     int ckpt_every, const float* w, InstanceView* out);

// FP64 per-cell gradient from the instance's accumulators, restricted to
// `level` into g (device pointer, or host pointer with MG_HOST_PTRS).
int finish_gradient(mg_mesh* mesh, int level, const double* eps_dev, double dt, int tiles,
                    double* g, int flags, void* stream);

}  // namespace mg
