// Host-side mesh builder: argument validation, FP64 P1 assembly (App. A),
// node reordering (reverse Cuthill-McKee or Morton), sliced-ELL layout,
// node/cell/facet incidence and the nesting maps (Sec. II-B).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "mg_internal.h"

namespace mg {
namespace {

// Measure |e| and gradients of the d+1 barycentric basis functions of a
// simplex with vertex coordinates X[(d+1)][d].  Returns false if degenerate.
bool simplex_geometry(int d, const double* X, double* vol, double* grad) {
  double E[3][3];  // E[r][k] = (x_{k+1} - x_0)_r
  for (int k = 0; k < d; ++k)
    for (int r = 0; r < d; ++r) E[r][k] = X[(k + 1) * d + r] - X[r];
  double inv[3][3];
  double det;
  if (d == 2) {
    det = E[0][0] * E[1][1] - E[0][1] * E[1][0];
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    inv[0][0] = E[1][1] / det;  inv[0][1] = -E[0][1] / det;
    inv[1][0] = -E[1][0] / det; inv[1][1] = E[0][0] / det;
    *vol = std::fabs(det) / 2.0;
  } else {
    const double c00 = E[1][1] * E[2][2] - E[1][2] * E[2][1];
    const double c01 = E[1][2] * E[2][0] - E[1][0] * E[2][2];
    const double c02 = E[1][0] * E[2][1] - E[1][1] * E[2][0];
    det = E[0][0] * c00 + E[0][1] * c01 + E[0][2] * c02;
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (E[0][2] * E[2][1] - E[0][1] * E[2][2]) / det;
    inv[1][1] = (E[0][0] * E[2][2] - E[0][2] * E[2][0]) / det;
    inv[2][1] = (E[0][1] * E[2][0] - E[0][0] * E[2][1]) / det;
    inv[0][2] = (E[0][1] * E[1][2] - E[0][2] * E[1][1]) / det;
    inv[1][2] = (E[0][2] * E[1][0] - E[0][0] * E[1][2]) / det;
    inv[2][2] = (E[0][0] * E[1][1] - E[0][1] * E[1][0]) / det;
    *vol = std::fabs(det) / 6.0;
  }
  // grad phi_{k+1} = row k of E^-1; grad phi_0 = -sum of the others
  for (int r = 0; r < d; ++r) grad[r] = 0.0;
  for (int k = 0; k < d; ++k)
    for (int r = 0; r < d; ++r) {
      grad[(k + 1) * d + r] = inv[k][r];
      grad[r] -= inv[k][r];
    }
  return true;
}

double facet_measure(int d, const double* coords, const int32_t* f) {
  if (d == 2) {
    const double* a = coords + 2 * (int64_t)f[0];
    const double* b = coords + 2 * (int64_t)f[1];
    return std::hypot(b[0] - a[0], b[1] - a[1]);
  }
  const double* a = coords + 3 * (int64_t)f[0];
  const double* b = coords + 3 * (int64_t)f[1];
  const double* c = coords + 3 * (int64_t)f[2];
  const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                       u[0] * v[1] - u[1] * v[0]};
  return 0.5 * std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
}

// Reverse Cuthill-McKee on the symmetric pattern (rowptr, col) of the
// caller-numbered stiffness.  Returns order[k] = node placed at row k.
std::vector<int32_t> rcm_order(int64_t n, const std::vector<int64_t>& rp,
                               const std::vector<int32_t>& ci) {
  std::vector<int32_t> deg(n);
  for (int64_t i = 0; i < n; ++i) deg[i] = (int32_t)(rp[i + 1] - rp[i]);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<char> seen(n, 0);
  std::vector<int32_t> level(n, -1);
  std::vector<int32_t> queue;
  queue.reserve(n);
  auto bfs = [&](int32_t s, std::vector<int32_t>& lv) {
    // returns the BFS queue (visit order) restricted to s's component
    queue.clear();
    queue.push_back(s);
    lv[s] = 0;
    for (size_t h = 0; h < queue.size(); ++h) {
      int32_t u = queue[h];
      for (int64_t k = rp[u]; k < rp[u + 1]; ++k) {
        int32_t v = ci[k];
        if (lv[v] < 0) { lv[v] = lv[u] + 1; queue.push_back(v); }
      }
    }
  };
  for (int64_t start_scan = 0; start_scan < n; ++start_scan) {
    if (seen[start_scan]) continue;
    // pseudo-peripheral start node (George-Liu): repeat BFS from the
    // min-degree node of the last level while the eccentricity grows
    int32_t s = (int32_t)start_scan;
    int ecc = -1;
    for (int it = 0; it < 8; ++it) {
      bfs(s, level);
      std::vector<int32_t> comp(queue);
      int e = level[comp.back()];
      int32_t best = comp.back();
      for (int32_t v : comp)
        if (level[v] == e && (deg[v] < deg[best] || (deg[v] == deg[best] && v < best)))
          best = v;
      for (int32_t v : comp) level[v] = -1;
      if (e <= ecc) break;
      ecc = e;
      s = best;
    }
    // Cuthill-McKee from s, neighbours by increasing degree then id
    size_t head = order.size();
    order.push_back(s);
    seen[s] = 1;
    std::vector<int32_t> nb;
    for (size_t h = head; h < order.size(); ++h) {
      int32_t u = order[h];
      nb.clear();
      for (int64_t k = rp[u]; k < rp[u + 1]; ++k)
        if (!seen[ci[k]]) nb.push_back(ci[k]);
      std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
      for (int32_t v : nb) { seen[v] = 1; order.push_back(v); }
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

uint64_t spread_bits2(uint64_t x) {  // 32 -> every other bit
  x &= 0xffffffffULL;
  x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
  x = (x | (x << 2)) & 0x3333333333333333ULL;
  x = (x | (x << 1)) & 0x5555555555555555ULL;
  return x;
}

uint64_t spread_bits3(uint64_t x) {  // 21 -> every third bit
  x &= 0x1fffffULL;
  x = (x | (x << 32)) & 0x1f00000000ffffULL;
  x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}

std::vector<int32_t> morton_order(int d, int64_t n, const double* X) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < n; ++i)
    for (int r = 0; r < d; ++r) {
      lo[r] = std::min(lo[r], X[i * d + r]);
      hi[r] = std::max(hi[r], X[i * d + r]);
    }
  double span = 0.0;
  for (int r = 0; r < d; ++r) span = std::max(span, hi[r] - lo[r]);
  if (!(span > 0.0)) span = 1.0;
  const double q = (d == 2 ? 4294967295.0 : 2097151.0) / span;
  std::vector<uint64_t> code(n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t c = 0;
    for (int r = 0; r < d; ++r) {
      uint64_t v = (uint64_t)((X[i * d + r] - lo[r]) * q);
      c |= (d == 2 ? spread_bits2(v) : spread_bits3(v)) << r;
    }
    code[i] = c;
  }
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return code[a] < code[b]; });
  return order;
}

}  // namespace

int build_host_mesh(int dim, int n_levels, const double* coords, int64_t n_nodes,
                    const int32_t* cells, int64_t n_cells,
                    const int32_t* const* cell_parent,
                    const int64_t* n_cells_per_level, const int32_t* bnd,
                    int64_t n_bnd, int bc_mode, int order, HostMesh& hm,
                    std::string& msg) {
  // ---- argument checks (no CUDA) ----------------------------------------
  if (dim != 2 && dim != 3) { msg = "dim must be 2 or 3"; return MG_ERR_ARG; }
  if (n_levels < 1 || n_levels > 16) { msg = "n_levels out of range"; return MG_ERR_ARG; }
  if (!coords || !cells || !n_cells_per_level) { msg = "null array"; return MG_ERR_ARG; }
  if (n_nodes < dim + 1 || n_nodes > 0x7fffffffLL) { msg = "n_nodes out of range"; return MG_ERR_ARG; }
  if (n_cells < 1 || n_cells > 0x7fffffffLL) { msg = "n_cells out of range"; return MG_ERR_ARG; }
  if (n_bnd < 0 || (n_bnd > 0 && !bnd)) { msg = "bad boundary facets"; return MG_ERR_ARG; }
  if (bc_mode < MG_BC_ABC1 || bc_mode > MG_BC_DIRICHLET) { msg = "bad bc_mode"; return MG_ERR_ARG; }
  if (order < MG_ORDER_RCM || order > MG_ORDER_NONE) { msg = "bad order"; return MG_ERR_ARG; }
  if (n_cells_per_level[n_levels - 1] != n_cells) {
    msg = "n_cells_per_level[last] != n_cells";
    return MG_ERR_ARG;
  }
  if (n_levels > 1 && !cell_parent) { msg = "cell_parent is null"; return MG_ERR_NESTING; }
  for (int l = 0; l < n_levels; ++l)
    if (n_cells_per_level[l] < 1) { msg = "empty level"; return MG_ERR_NESTING; }
  for (int64_t i = 0; i < n_nodes * dim; ++i)
    if (!std::isfinite(coords[i])) { msg = "non-finite coordinate"; return MG_ERR_ARG; }
  const int k = dim + 1;
  for (int64_t c = 0; c < n_cells; ++c)
    for (int a = 0; a < k; ++a) {
      int32_t v = cells[c * k + a];
      if (v < 0 || v >= n_nodes) { msg = "cell node id out of range"; return MG_ERR_ARG; }
      for (int b = 0; b < a; ++b)
        if (cells[c * k + b] == v) { msg = "repeated node in a cell"; return MG_ERR_ARG; }
    }
  for (int64_t f = 0; f < n_bnd * dim; ++f)
    if (bnd[f] < 0 || bnd[f] >= n_nodes) { msg = "facet node id out of range"; return MG_ERR_ARG; }

  // nesting maps -> ancestors of each finest cell on every level
  hm.ancestors.assign(n_levels, {});
  hm.ancestors[n_levels - 1].resize(n_cells);
  std::iota(hm.ancestors[n_levels - 1].begin(), hm.ancestors[n_levels - 1].end(), 0);
  for (int l = n_levels - 1; l >= 1; --l) {
    const int32_t* par = cell_parent[l - 1];
    const int64_t nc = n_cells_per_level[l], np = n_cells_per_level[l - 1];
    if (!par) { msg = "cell_parent level missing"; return MG_ERR_NESTING; }
    std::vector<int32_t> cnt(np, 0);
    for (int64_t c = 0; c < nc; ++c) {
      if (par[c] < 0 || par[c] >= np) { msg = "parent id out of range"; return MG_ERR_NESTING; }
      cnt[par[c]]++;
    }
    for (int64_t p = 0; p < np; ++p)
      if (cnt[p] == 0) { msg = "coarse cell without children"; return MG_ERR_NESTING; }
    auto& dst = hm.ancestors[l - 1];
    const auto& src = hm.ancestors[l];
    dst.resize(n_cells);
    for (int64_t e = 0; e < n_cells; ++e) dst[e] = par[src[e]];
  }

  hm.dim = dim;
  hm.n_levels = n_levels;
  hm.bc = bc_mode;
  hm.n = n_nodes;
  hm.m = n_cells;
  hm.nb = n_bnd;
  hm.n_cells_level.assign(n_cells_per_level, n_cells_per_level + n_levels);

  // ---- geometry and element stiffness ------------------------------------
  hm.cell_vol.resize(n_cells);
  std::vector<double> Ke((size_t)n_cells * k * k);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t c = 0; c < n_cells; ++c) {
    double X[12], G[12], vol;
    for (int a = 0; a < k; ++a)
      for (int r = 0; r < dim; ++r) X[a * dim + r] = coords[(int64_t)cells[c * k + a] * dim + r];
    if (!simplex_geometry(dim, X, &vol, G)) { bad++; continue; }
    hm.cell_vol[c] = vol;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double s = 0.0;
        for (int r = 0; r < dim; ++r) s += G[a * dim + r] * G[b * dim + r];
        Ke[((size_t)c * k + a) * k + b] = vol * s;
      }
  }
  if (bad) { msg = "degenerate cell"; return MG_ERR_ARG; }

  // node -> cells incidence (caller numbering)
  std::vector<int64_t> ncp(n_nodes + 1, 0);
  for (int64_t i = 0; i < n_cells * k; ++i) ncp[cells[i] + 1]++;
  for (int64_t i = 0; i < n_nodes; ++i) {
    if (ncp[i + 1] == 0) { msg = "node not used by any cell"; return MG_ERR_ARG; }
    ncp[i + 1] += ncp[i];
  }
  std::vector<int32_t> ncc(ncp[n_nodes]);
  std::vector<int8_t> ncl(ncp[n_nodes]);  // local vertex index in the cell
  {
    std::vector<int64_t> fill(ncp.begin(), ncp.end() - 1);
    for (int64_t c = 0; c < n_cells; ++c)
      for (int a = 0; a < k; ++a) {
        int64_t pos = fill[cells[c * k + a]]++;
        ncc[pos] = (int32_t)c;
        ncl[pos] = (int8_t)a;
      }
  }

  // stiffness pattern + values in caller numbering (row i gathers from its cells)
  std::vector<int64_t> rp(n_nodes + 1, 0);
  std::vector<std::vector<int32_t>> rows_col(n_nodes);
  std::vector<std::vector<double>> rows_val(n_nodes);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n_nodes; ++i) {
    auto& cs = rows_col[i];
    for (int64_t q = ncp[i]; q < ncp[i + 1]; ++q) {
      const int32_t c = ncc[q];
      for (int b = 0; b < k; ++b) cs.push_back(cells[(int64_t)c * k + b]);
    }
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    auto& vs = rows_val[i];
    vs.assign(cs.size(), 0.0);
    for (int64_t q = ncp[i]; q < ncp[i + 1]; ++q) {
      const int32_t c = ncc[q];
      const int a = ncl[q];
      for (int b = 0; b < k; ++b) {
        const int32_t j = cells[(int64_t)c * k + b];
        const size_t pos = std::lower_bound(cs.begin(), cs.end(), j) - cs.begin();
        vs[pos] += Ke[((size_t)c * k + a) * k + b];
      }
    }
  }
  std::vector<double>().swap(Ke);
  for (int64_t i = 0; i < n_nodes; ++i) rp[i + 1] = rp[i] + (int64_t)rows_col[i].size();
  std::vector<int32_t> ci(rp[n_nodes]);
  for (int64_t i = 0; i < n_nodes; ++i)
    std::copy(rows_col[i].begin(), rows_col[i].end(), ci.begin() + rp[i]);

  // ---- node order ---------------------------------------------------------
  std::vector<int32_t> ord;
  if (order == MG_ORDER_RCM) ord = rcm_order(n_nodes, rp, ci);
  else if (order == MG_ORDER_MORTON) ord = morton_order(dim, n_nodes, coords);
  else { ord.resize(n_nodes); std::iota(ord.begin(), ord.end(), 0); }
  hm.iperm = ord;
  hm.perm.assign(n_nodes, -1);
  for (int64_t r = 0; r < n_nodes; ++r) hm.perm[ord[r]] = (int32_t)r;
  hm.coords.resize((size_t)n_nodes * dim);
  for (int64_t r = 0; r < n_nodes; ++r)
    for (int a = 0; a < dim; ++a) hm.coords[(size_t)r * dim + a] = coords[(size_t)ord[r] * dim + a];

  // ---- stiffness in row order, diagonal first -----------------------------
  hm.rowptr.assign(n_nodes + 1, 0);
  for (int64_t r = 0; r < n_nodes; ++r)
    hm.rowptr[r + 1] = hm.rowptr[r] + (int64_t)rows_col[ord[r]].size();
  hm.col.resize(hm.rowptr[n_nodes]);
  hm.val.resize(hm.rowptr[n_nodes]);
  hm.row_abs.assign(n_nodes, 0.0);
  int maxnz = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(max : maxnz)
  for (int64_t r = 0; r < n_nodes; ++r) {
    const int32_t i = ord[r];
    const auto& cs = rows_col[i];
    const auto& vs = rows_val[i];
    std::vector<std::pair<int32_t, double>> e(cs.size());
    for (size_t t = 0; t < cs.size(); ++t) e[t] = {hm.perm[cs[t]], vs[t]};
    std::sort(e.begin(), e.end(), [&](const auto& a, const auto& b) {
      const bool da = a.first == (int32_t)r, db = b.first == (int32_t)r;
      if (da != db) return da;
      return a.first < b.first;
    });
    double s = 0.0;
    for (size_t t = 0; t < e.size(); ++t) {
      hm.col[hm.rowptr[r] + t] = e[t].first;
      hm.val[hm.rowptr[r] + t] = e[t].second;
      s += std::fabs(e[t].second);
    }
    hm.row_abs[r] = s;
    maxnz = std::max(maxnz, (int)e.size());
  }
  hm.max_row_nnz = maxnz;
  std::vector<std::vector<int32_t>>().swap(rows_col);
  std::vector<std::vector<double>>().swap(rows_val);

  // ---- sliced ELL ---------------------------------------------------------
  hm.n_slices = (n_nodes + kSliceH - 1) / kSliceH;
  hm.slice_off.assign(hm.n_slices + 1, 0);
  hm.slice_w.assign(hm.n_slices, 0);
  for (int64_t s = 0; s < hm.n_slices; ++s) {
    int w = 0;
    for (int64_t r = s * kSliceH; r < std::min<int64_t>(n_nodes, (s + 1) * kSliceH); ++r)
      w = std::max<int>(w, (int)(hm.rowptr[r + 1] - hm.rowptr[r]));
    hm.slice_w[s] = w;
    hm.slice_off[s + 1] = hm.slice_off[s] + (int64_t)w * kSliceH;
  }
  hm.ell.resize(hm.slice_off[hm.n_slices]);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < hm.n_slices; ++s) {
    const int w = hm.slice_w[s];
    for (int rl = 0; rl < kSliceH; ++rl) {
      const int64_t r = s * kSliceH + rl;
      const int64_t valid_row = std::min<int64_t>(r, n_nodes - 1);
      const int64_t nz = r < n_nodes ? hm.rowptr[r + 1] - hm.rowptr[r] : 0;
      for (int t = 0; t < w; ++t) {
        EllEntry e;
        if (t < nz) {
          e.col = hm.col[hm.rowptr[r] + t];
          e.val = (float)hm.val[hm.rowptr[r] + t];
        } else {
          e.col = (int32_t)valid_row;
          e.val = 0.0f;
        }
        hm.ell[hm.slice_off[s] + (int64_t)t * kSliceH + rl] = e;
      }
    }
  }

  // ---- cells and incidence in row numbering --------------------------------
  hm.cells.resize((size_t)n_cells * k);
  for (int64_t i = 0; i < n_cells * k; ++i) hm.cells[i] = hm.perm[cells[i]];
  hm.nc_ptr.assign(n_nodes + 1, 0);
  for (int64_t r = 0; r < n_nodes; ++r)
    hm.nc_ptr[r + 1] = hm.nc_ptr[r] + (ncp[ord[r] + 1] - ncp[ord[r]]);
  hm.nc_cell.resize(hm.nc_ptr[n_nodes]);
  hm.nc_w.resize(hm.nc_ptr[n_nodes]);
  for (int64_t r = 0; r < n_nodes; ++r) {
    const int32_t i = ord[r];
    int64_t o = hm.nc_ptr[r];
    for (int64_t q = ncp[i]; q < ncp[i + 1]; ++q, ++o) {
      hm.nc_cell[o] = ncc[q];
      hm.nc_w[o] = hm.cell_vol[ncc[q]] / k;
    }
  }

  // ---- boundary facets: owner cell and measure -----------------------------
  hm.bnd.resize((size_t)n_bnd * dim);
  hm.bnd_owner.resize(n_bnd);
  hm.bnd_meas.resize(n_bnd);
  hm.is_bnd_row.assign(n_nodes, 0);
  for (int64_t f = 0; f < n_bnd; ++f) {
    const int32_t* fv = bnd + f * dim;
    int owner = -1, count = 0;
    for (int64_t q = ncp[fv[0]]; q < ncp[fv[0] + 1]; ++q) {
      const int32_t c = ncc[q];
      int hit = 0;
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < k; ++b)
          if (cells[(int64_t)c * k + b] == fv[a]) { hit++; break; }
      if (hit == dim) { owner = c; count++; }
    }
    if (count != 1) { msg = "boundary facet is not a facet of exactly one cell"; return MG_ERR_ARG; }
    hm.bnd_owner[f] = owner;
    hm.bnd_meas[f] = facet_measure(dim, coords, fv);
    for (int a = 0; a < dim; ++a) {
      hm.bnd[f * dim + a] = hm.perm[fv[a]];
      hm.is_bnd_row[hm.perm[fv[a]]] = 1;
    }
  }
  hm.nf_ptr.assign(n_nodes + 1, 0);
  for (int64_t f = 0; f < n_bnd * dim; ++f) hm.nf_ptr[hm.bnd[f] + 1]++;
  for (int64_t r = 0; r < n_nodes; ++r) hm.nf_ptr[r + 1] += hm.nf_ptr[r];
  hm.nf_cell.resize(hm.nf_ptr[n_nodes]);
  hm.nf_w.resize(hm.nf_ptr[n_nodes]);
  {
    std::vector<int64_t> fill(hm.nf_ptr.begin(), hm.nf_ptr.end() - 1);
    for (int64_t f = 0; f < n_bnd; ++f)
      for (int a = 0; a < dim; ++a) {
        const int64_t pos = fill[hm.bnd[f * dim + a]]++;
        hm.nf_cell[pos] = hm.bnd_owner[f];
        hm.nf_w[pos] = hm.bnd_meas[f] / dim;
      }
  }
  return MG_OK;
}

int build_tiles(const HostMesh& hm, int P, HostTiles& T) {
  if (P <= 0 || P % kSliceH != 0 || P > 8192) return MG_ERR_ARG;
  const int64_t n = hm.n;
  T.P = P;
  T.n_tiles = (n + P - 1) / P;
  const int64_t spt = P / kSliceH;  // slices per tile
  T.ell_off.assign(T.n_tiles + 1, 0);
  T.halo_off.assign(T.n_tiles + 1, 0);
  T.halo_cnt.assign(T.n_tiles, 0);
  T.slice_info.assign(2 * hm.n_slices, 0);
  std::vector<std::vector<int32_t>> halos(T.n_tiles);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
  for (int64_t t = 0; t < T.n_tiles; ++t) {
    const int64_t r0 = t * P, r1 = std::min<int64_t>(n, r0 + P);
    auto& h = halos[t];
    for (int64_t r = r0; r < r1; ++r)
      for (int64_t q = hm.rowptr[r]; q < hm.rowptr[r + 1]; ++q)
        if (hm.col[q] < r0 || hm.col[q] >= r1) h.push_back(hm.col[q]);
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    if ((int64_t)P + (int64_t)h.size() > 65535) bad++;
  }
  if (bad) return MG_ERR_ARG;
  int64_t total_rows = 0;
  for (int64_t t = 0; t < T.n_tiles; ++t) {
    const int64_t r0 = t * P, r1 = std::min<int64_t>(n, r0 + P);
    T.halo_cnt[t] = (int32_t)halos[t].size();
    T.halo_off[t + 1] = T.halo_off[t] + (halos[t].size() + 3) / 4 * 4;
    int64_t e = 0;
    for (int64_t s = t * spt; s < std::min<int64_t>(hm.n_slices, (t + 1) * spt); ++s) {
      T.slice_info[2 * s] = (int32_t)e;
      T.slice_info[2 * s + 1] = hm.slice_w[s];
      e += (int64_t)hm.slice_w[s] * kSliceH;
    }
    e = (e + 7) / 8 * 8;
    T.ell_off[t + 1] = T.ell_off[t] + e;
    T.max_ell = std::max<int>(T.max_ell, (int)e);
    T.max_halo = std::max<int>(T.max_halo, (int)(T.halo_off[t + 1] - T.halo_off[t]));
    total_rows += (r1 - r0) + (int64_t)halos[t].size();
  }
  T.halo_ratio = (double)total_rows / (double)n;
  T.halo.assign(T.halo_off[T.n_tiles], 0);
  T.ell_idx.assign(T.ell_off[T.n_tiles], 0);
  T.ell_val.assign(T.ell_off[T.n_tiles], 0.0f);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < T.n_tiles; ++t) {
    const int64_t r0 = t * P, r1 = std::min<int64_t>(n, r0 + P);
    const auto& h = halos[t];
    std::copy(h.begin(), h.end(), T.halo.begin() + T.halo_off[t]);
    // halo rows follow the tile's own rows (r1 - r0 of them; fewer than P
    // in the last tile), matching the order in which they are staged
    auto local = [&](int32_t c) -> uint16_t {
      if (c >= r0 && c < r1) return (uint16_t)(c - r0);
      return (uint16_t)((r1 - r0) + (std::lower_bound(h.begin(), h.end(), c) - h.begin()));
    };
    for (int64_t s = t * spt; s < std::min<int64_t>(hm.n_slices, (t + 1) * spt); ++s) {
      const int w = hm.slice_w[s];
      const int64_t base = T.ell_off[t] + T.slice_info[2 * s];
      for (int rl = 0; rl < kSliceH; ++rl) {
        const int64_t r = s * kSliceH + rl;
        const int64_t vr = std::min<int64_t>(r, r1 - 1);  // padding rows point at a valid row
        const int64_t nz = r < r1 ? hm.rowptr[r + 1] - hm.rowptr[r] : 0;
        for (int k = 0; k < w; ++k) {
          uint16_t li;
          float v;
          if (k < nz) {
            li = local(hm.col[hm.rowptr[r] + k]);
            v = (float)hm.val[hm.rowptr[r] + k];
          } else {
            li = (uint16_t)(vr - r0);
            v = 0.0f;
          }
          T.ell_idx[base + (int64_t)k * kSliceH + rl] = li;
          T.ell_val[base + (int64_t)k * kSliceH + rl] = v;
        }
      }
    }
  }
  return MG_OK;
}

void level_children(const HostMesh& hm, int level, std::vector<int64_t>& ptr,
                    std::vector<int32_t>& idx) {
  const auto& anc = hm.ancestors[level];
  const int64_t nc = hm.n_cells_level[level];
  ptr.assign(nc + 1, 0);
  for (int64_t e = 0; e < hm.m; ++e) ptr[anc[e] + 1]++;
  for (int64_t c = 0; c < nc; ++c) ptr[c + 1] += ptr[c];
  idx.resize(hm.m);
  std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t e = 0; e < hm.m; ++e) idx[fill[anc[e]]++] = (int32_t)e;
}

}  // namespace mg
