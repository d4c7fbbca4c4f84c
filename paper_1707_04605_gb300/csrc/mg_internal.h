// Internal declarations shared by the host mesh builder and the CUDA side.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mgwave.h"

namespace mg {

// Rows of the sliced-ELL stiffness are grouped in slices of this height;
// inside a slice, entry k of row r sits at slice_off + k * kSliceH + r
// (column-major), so a warp working on consecutive rows of one slice reads
// entry k of all its rows from one contiguous span.  The diagonal is entry
// 0 of every row; padding entries point at the row itself with value 0.
constexpr int kSliceH = 32;

struct EllEntry {       // 8 bytes, loaded as int2 on the device
  int32_t col;
  float val;
};

// Host-side image of a mesh, node-indexed arrays in internal row order.
struct HostMesh {
  int dim = 0;
  int n_levels = 0;
  int bc = MG_BC_ABC1;
  int64_t n = 0;        // nodes
  int64_t m = 0;        // finest cells
  int64_t nb = 0;       // boundary facets
  std::vector<int64_t> n_cells_level;

  std::vector<int32_t> perm;   // caller node -> row
  std::vector<int32_t> iperm;  // row -> caller node
  std::vector<double> coords;  // [n][dim] node coordinates, rows

  // stiffness (rows/cols internal, diagonal first), FP64
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<double> row_abs;  // sum_j |K_ij| per row
  int max_row_nnz = 0;

  // sliced ELL
  int64_t n_slices = 0;
  std::vector<int64_t> slice_off;   // [n_slices + 1]
  std::vector<int32_t> slice_w;     // [n_slices]
  std::vector<EllEntry> ell;

  // node (row) -> incident finest cells, weight |e|/(d+1)
  std::vector<int64_t> nc_ptr;
  std::vector<int32_t> nc_cell;
  std::vector<double> nc_w;
  // node (row) -> incident boundary facets: owner cell, weight |F|/d
  std::vector<int64_t> nf_ptr;
  std::vector<int32_t> nf_cell;
  std::vector<double> nf_w;

  std::vector<double> cell_vol;     // |e|, caller cell order
  std::vector<int32_t> cells;       // [m][dim+1], rows (internal node ids)
  std::vector<int32_t> bnd;         // [nb][dim], rows
  std::vector<int32_t> bnd_owner;   // [nb]
  std::vector<double> bnd_meas;     // |F|
  std::vector<int32_t> is_bnd_row;  // [n] 1 if the row is on a boundary facet

  // nesting: ancestors[l][e] = level-l ancestor of finest cell e
  std::vector<std::vector<int32_t>> ancestors;
};

// Builds the host image; returns MG_OK or an MG_ERR_* code and a message.
int build_host_mesh(int dim, int n_levels, const double* coords, int64_t n_nodes,
                    const int32_t* cells, int64_t n_cells,
                    const int32_t* const* cell_parent,
                    const int64_t* n_cells_per_level, const int32_t* bnd,
                    int64_t n_bnd, int bc_mode, int order, HostMesh& out,
                    std::string& msg);

// Level cell -> finest cells CSR for the restriction (deterministic order).
void level_children(const HostMesh& hm, int level, std::vector<int64_t>& ptr,
                    std::vector<int32_t>& idx);

// Row tiles for shared-memory staging.  Tile t owns rows [t*P, t*P + P) (P a
// multiple of kSliceH).  Its halo is the sorted list of rows outside that
// range that its stiffness rows reference.  The tile's stiffness entries are
// re-indexed locally: index i < P_t is row t*P + i, index P_t + h is halo
// row h, where P_t = min(P, n - t*P) is the tile's own row count.
// Per tile, the entries of its slices are stored contiguously (same
// column-major slice layout as the global ELL), padded to a multiple of 8
// entries so that 16-byte copies can stage them.
struct HostTiles {
  int P = 0;
  int64_t n_tiles = 0;
  std::vector<int64_t> ell_off;     // [n_tiles+1] entry offset of each tile
  std::vector<uint16_t> ell_idx;    // local indices
  std::vector<float> ell_val;
  std::vector<int32_t> slice_info;  // [n_slices][2]: {offset within tile, width}
  std::vector<int64_t> halo_off;    // [n_tiles+1], padded to multiples of 4
  std::vector<int32_t> halo_cnt;    // [n_tiles] real halo sizes
  std::vector<int32_t> halo;        // global rows
  int max_ell = 0;                  // max entries of a tile (padded)
  int max_halo = 0;                 // max halo rows of a tile (padded)
  double halo_ratio = 0.0;          // (sum of tile rows + halo rows) / n
};

// Returns MG_ERR_ARG if P is not a positive multiple of kSliceH or a tile's
// local index space (P + halo) does not fit 16 bits.
int build_tiles(const HostMesh& hm, int P, HostTiles& out);

}  // namespace mg
