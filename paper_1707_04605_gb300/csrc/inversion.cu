// TV-regularised reconstruction (Sec. II: reconstruction procedure, coarse-
// to-fine approach, compression of coefficients) on top of the exact
// Jacobian products of the library.
//
// The linearised model y - y0 = L x + n (x: perturbation of the level-cell
// permittivity values, x0 = 0) is inverted by the iteration (tv_iteration)
//   x_{l+1} = (L^T L + alpha D^T G_l D)^{-1} L^T (y - y0),
//   G_0 = I,  G_l = diag(|D x_l|)^{-1}  (entries below 1e-8 max|D x_l| raised),
// with D of (d_mat): D_ij = -s_ij / s_max (s_ij the measure of the boundary
// shared by cells i and j), D_ii = beta + sum_j s_ij / s_max.  Every linear
// system is solved matrix-free by conjugate gradients in FP64 (inner
// products included); L v is mg_jacobian_apply, L^T w is
// mg_jacobian_T_apply on checkpoints written once (or, for projected data,
// the same composed with mg_project / mg_projected_weights).
//
// Coarse-to-fine with two nested levels c < f, steps (1)-(5): a coarse
// update on level c (tv_iteration_0), then a fine correction (tv_iteration_2)
// in the coordinates of the fine fluctuations.  The basis of the
// fluctuations inside a coarse cell joins adjacent children (+1 / -1) along
// a breadth-first spanning tree of the children's facet adjacency, rooted
// at the child with the most sibling neighbours (ties: lowest index); in 2D
// these are the centre-corner pairs of Sec. II.  L_f = L R_f and
// D_f = D_level_f R_f.  Compression keeps the basis functions of the
// ceil(keep_frac n_c) coarse cells with the largest |x_c| (ties: lower
// index); the fine system is solved on that subspace (a 0/1 mask).
//
// More nested levels l_0 < l_1 < ... < l_nf (tv_iteration_3): after the
// coarse update, each f_i (the fluctuations of level l_i inside the cells
// of l_{i-1}) gets a compressed correction against the data that the
// coarse update and the corrections of f_1..f_{i-1} of the same outer step
// leave.  Those are assembled on the cells of l_{i-1} (comp: each cell
// takes its parent's value plus its own fluctuation), so the residual is
// dy - J_{l_{i-1}} comp, one Jacobian product; compression ranks the cells
// of l_{i-1} by |comp|.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/mgwave.h"
#include "mesh_view.h"
#include "mg_internal.h"

namespace mg {
namespace {

// ------------------------------------------------------------------ host
struct Csr {
  int64_t n = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
  std::vector<double> val;
};

double facet_measure(const HostMesh& hm, const int32_t* v) {
  const double* X = hm.coords.data();
  if (hm.dim == 2) {
    const double dx = X[2 * v[1]] - X[2 * v[0]], dy = X[2 * v[1] + 1] - X[2 * v[0] + 1];
    return std::sqrt(dx * dx + dy * dy);
  }
  double a[3], b[3];
  for (int i = 0; i < 3; ++i) {
    a[i] = X[3 * v[1] + i] - X[3 * v[0] + i];
    b[i] = X[3 * v[2] + i] - X[3 * v[0] + i];
  }
  const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2],
               cz = a[0] * b[1] - a[1] * b[0];
  return 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
}

// Interior facets of the finest mesh: the cells on both sides and the
// facet measure (facets are matched by sorting their node triples).
struct Facets {
  std::vector<int32_t> a, b;
  std::vector<double> meas;
};

int interior_facets(const HostMesh& hm, Facets& out) {
  const int d = hm.dim, k = d + 1;
  struct Key {
    std::array<int32_t, 3> v;
    int32_t cell;
  };
  std::vector<Key> keys((size_t)hm.m * k);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < hm.m; ++e) {
    const int32_t* c = hm.cells.data() + (size_t)e * k;
    for (int f = 0; f < k; ++f) {
      Key key;
      key.v = {-1, -1, -1};
      int t = 0;
      for (int j = 0; j < k; ++j)
        if (j != f) key.v[t++] = c[j];
      std::sort(key.v.begin(), key.v.begin() + d);
      key.cell = (int32_t)e;
      keys[(size_t)e * k + f] = key;
    }
  }
  std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
    return x.v != y.v ? x.v < y.v : x.cell < y.cell;
  });
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].v == keys[i].v) ++j;
    if (j - i > 2) return MG_ERR_ARG;  // a facet of more than two cells
    if (j - i == 2) {
      out.a.push_back(keys[i].cell);
      out.b.push_back(keys[i + 1].cell);
      out.meas.push_back(facet_measure(hm, keys[i].v.data()));
    }
    i = j;
  }
  return MG_OK;
}

// Shared-boundary measures between the cells of `level` (symmetric CSR,
// columns ascending, no diagonal).
Csr level_graph(const HostMesh& hm, const Facets& F, int level) {
  const auto& anc = hm.ancestors[level];
  struct P {
    int32_t i, j;
    double s;
  };
  std::vector<P> pairs;
  for (size_t q = 0; q < F.a.size(); ++q) {
    const int32_t A = anc[F.a[q]], B = anc[F.b[q]];
    if (A == B) continue;
    pairs.push_back({A, B, F.meas[q]});
    pairs.push_back({B, A, F.meas[q]});
  }
  std::sort(pairs.begin(), pairs.end(),
            [](const P& x, const P& y) { return x.i != y.i ? x.i < y.i : x.j < y.j; });
  Csr g;
  g.n = hm.n_cells_level[level];
  g.ptr.assign(g.n + 1, 0);
  for (size_t q = 0; q < pairs.size();) {
    size_t r = q;
    double s = 0.0;
    while (r < pairs.size() && pairs[r].i == pairs[q].i && pairs[r].j == pairs[q].j)
      s += pairs[r++].s;
    g.idx.push_back(pairs[q].j);
    g.val.push_back(s);
    g.ptr[pairs[q].i + 1]++;
    q = r;
  }
  for (int64_t i = 0; i < g.n; ++i) g.ptr[i + 1] += g.ptr[i];
  return g;
}

// D of (d_mat) from a level graph (diagonal first in every row).
Csr reg_matrix(const Csr& g, double beta) {
  double smax = 0.0;
  for (double s : g.val) smax = std::max(smax, s);
  if (smax <= 0.0) smax = 1.0;
  Csr D;
  D.n = g.n;
  D.ptr.assign(g.n + 1, 0);
  for (int64_t i = 0; i < g.n; ++i) {
    double sum = 0.0;
    for (int64_t q = g.ptr[i]; q < g.ptr[i + 1]; ++q) sum += g.val[q];
    D.idx.push_back((int32_t)i);
    D.val.push_back(beta + sum / smax);
    for (int64_t q = g.ptr[i]; q < g.ptr[i + 1]; ++q) {
      D.idx.push_back(g.idx[q]);
      D.val.push_back(-g.val[q] / smax);
    }
    D.ptr[i + 1] = (int64_t)D.idx.size();
  }
  return D;
}

bool adjacent(const Csr& g, int32_t a, int32_t b) {
  return std::binary_search(g.idx.begin() + g.ptr[a], g.idx.begin() + g.ptr[a + 1], b);
}

// Fine-fluctuation basis: plus/minus level-f cells and coarse cell per
// function, and the per-cell incidence CSR {basis index, sign}.
struct Basis {
  std::vector<int32_t> plus, minus, coarse;
  std::vector<int64_t> cptr;   // [n_f + 1]
  std::vector<int32_t> cfun;   // basis index
  std::vector<double> csign;   // +1 / -1
};

int fine_basis(const Csr& gf, const std::vector<int32_t>& parent, int64_t n_c, Basis& B) {
  const int64_t n_f = (int64_t)parent.size();
  std::vector<std::vector<int32_t>> kids(n_c);
  for (int64_t e = 0; e < n_f; ++e) kids[parent[e]].push_back((int32_t)e);
  std::vector<char> seen(n_f, 0);
  for (int64_t c = 0; c < n_c; ++c) {
    const auto& K = kids[c];
    if (K.empty()) return MG_ERR_NESTING;
    int best = -1;
    int32_t root = K[0];
    for (int32_t a : K) {
      int deg = 0;
      for (int32_t b : K)
        if (b != a && adjacent(gf, a, b)) ++deg;
      if (deg > best) { best = deg; root = a; }
    }
    std::vector<int32_t> queue{root};
    seen[root] = 1;
    for (size_t h = 0; h < queue.size(); ++h) {
      const int32_t a = queue[h];
      for (int32_t b : K)
        if (!seen[b] && adjacent(gf, a, b)) {
          B.plus.push_back(b);
          B.minus.push_back(a);
          B.coarse.push_back((int32_t)c);
          seen[b] = 1;
          queue.push_back(b);
        }
    }
    if (queue.size() != K.size()) return MG_ERR_NESTING;  // children not facet-connected
  }
  B.cptr.assign(n_f + 1, 0);
  for (size_t k = 0; k < B.plus.size(); ++k) {
    B.cptr[B.plus[k] + 1]++;
    B.cptr[B.minus[k] + 1]++;
  }
  for (int64_t e = 0; e < n_f; ++e) B.cptr[e + 1] += B.cptr[e];
  B.cfun.resize(B.cptr[n_f]);
  B.csign.resize(B.cptr[n_f]);
  std::vector<int64_t> fill(B.cptr.begin(), B.cptr.end() - 1);
  for (size_t k = 0; k < B.plus.size(); ++k) {
    B.cfun[fill[B.plus[k]]] = (int32_t)k;
    B.csign[fill[B.plus[k]]++] = 1.0;
    B.cfun[fill[B.minus[k]]] = (int32_t)k;
    B.csign[fill[B.minus[k]]++] = -1.0;
  }
  return MG_OK;
}

// ---------------------------------------------------------------- device
constexpr int kRed = 1024;

// out[0] = sum x_i y_i (one block, fixed reduction order)
__global__ void __launch_bounds__(kRed) k_dot(int64_t n, const double* x, const double* y,
                                              double* out) {
  __shared__ double sh[kRed];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kRed) s += x[i] * y[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRed / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

__global__ void __launch_bounds__(kRed) k_max_abs(int64_t n, const double* x, double* out) {
  __shared__ double sh[kRed];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kRed) s = fmax(s, fabs(x[i]));
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRed / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

#define MG_GRID_LOOP(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// out = a x + b y  (y may be null when b = 0)
__global__ void k_lincomb(int64_t n, double a, const double* x, double b, const double* y,
                          double* out) {
  MG_GRID_LOOP(i, n) out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// out = A x for a CSR matrix (FP64)
__global__ void k_csr(int64_t n, const int64_t* ptr, const int32_t* idx, const double* val,
                      const double* x, double* out) {
  MG_GRID_LOOP(i, n) {
    double s = 0.0;
    for (int64_t q = ptr[i]; q < ptr[i + 1]; ++q) s += val[q] * x[idx[q]];
    out[i] = s;
  }
}

// g = 1 / max(|t|, 1e-8 tmax), or 1 on the first step or while tmax = 0
__global__ void k_weights(int64_t n, const double* t, const double* tmax, int first, double* g) {
  const double m = *tmax;
  MG_GRID_LOOP(i, n) g[i] = (first || m == 0.0) ? 1.0 : 1.0 / fmax(fabs(t[i]), 1e-8 * m);
}

__global__ void k_mul(int64_t n, const double* g, double* t) { MG_GRID_LOOP(i, n) t[i] *= g[i]; }

// cells[e] = sum over the basis functions at cell e of sign * v_k (mask applied)
__global__ void k_rf(int64_t n_f, const int64_t* ptr, const int32_t* fun, const double* sign,
                     const double* mask, const double* v, double* cells) {
  MG_GRID_LOOP(e, n_f) {
    double s = 0.0;
    for (int64_t q = ptr[e]; q < ptr[e + 1]; ++q) s += sign[q] * mask[fun[q]] * v[fun[q]];
    cells[e] = s;
  }
}

// v_k = mask_k (g[plus_k] - g[minus_k])
__global__ void k_rft(int64_t n_b, const int32_t* plus, const int32_t* minus, const double* mask,
                      const double* g, double* v) {
  MG_GRID_LOOP(k, n_b) v[k] = mask[k] * (g[plus[k]] - g[minus[k]]);
}

// out[e] = xc[parent[e]] + cells[e]
__global__ void k_level_sum(int64_t n_f, const int32_t* parent, const double* xc,
                            const double* cells, double* out) {
  MG_GRID_LOOP(e, n_f) out[e] = xc[parent[e]] + (cells ? cells[e] : 0.0);
}

__global__ void k_sub_f(int64_t n, const float* a, const float* b, float* out) {
  MG_GRID_LOOP(i, n) out[i] = a[i] - b[i];
}
__global__ void k_sub_d(int64_t n, const double* a, const double* b, double* out) {
  MG_GRID_LOOP(i, n) out[i] = a[i] - b[i];
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// ----------------------------------------------------------------- solver
struct DevCsr {
  int64_t n = 0;
  int64_t* ptr = nullptr;
  int32_t* idx = nullptr;
  double* val = nullptr;
};

struct Arena {  // stream-ordered device scratch, released with the solver
  cudaStream_t st;
  std::vector<void*> blocks;
  explicit Arena(cudaStream_t s) : st(s) {}
  ~Arena() {
    for (void* p : blocks) cudaFreeAsync(p, st);
  }
  template <class T>
  int get(T** out, size_t count) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(T), st) != cudaSuccess)
      return MG_ERR_OOM;
    blocks.push_back(p);
    *out = static_cast<T*>(p);
    return MG_OK;
  }
  template <class T>
  int put(T** out, const std::vector<T>& v) {
    int rc = get(out, v.size());
    if (rc) return rc;
    if (!v.empty() &&
        cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return MG_ERR_CUDA;
    return MG_OK;
  }
  int put_csr(DevCsr& d, const Csr& h) {
    d.n = h.n;
    int rc = put(&d.ptr, h.ptr);
    if (!rc) rc = put(&d.idx, h.idx);
    if (!rc) rc = put(&d.val, h.val);
    return rc;
  }
};

#define MG_RC(x)                  \
  do {                            \
    const int rc_ = (x);          \
    if (rc_ != MG_OK) return rc_; \
  } while (0)
#define MG_CK(x) \
  do {           \
    if ((x) != cudaSuccess) return MG_ERR_CUDA; \
  } while (0)

struct Solver {
  mg_mesh* M;
  const double* eps;
  const mg_shots* shots;
  const double* wav;
  double dt;
  int nt;
  int mode;
  const void* dy;     // device
  const float* u;     // device (projected mode)
  mg_tv_params P;
  cudaStream_t st;
  int fl;             // flags for the inner calls
  int64_t R = 0;
  Arena* A = nullptr;
  float* tr = nullptr;     // [R][nt] traces scratch
  float* tr2 = nullptr;    // [R][nt] traces scratch
  double* pd = nullptr;    // [2][R] projected scratch
  double* pd2 = nullptr;
  double* red = nullptr;   // reduction outputs
  int64_t launches = 0;

  int64_t data_len() const { return mode == MG_DATA_PROJECTED ? 2 * R : R * nt; }

  int dot(int64_t n, const double* x, const double* y, double* out) {
    k_dot<<<1, kRed, 0, st>>>(n, x, y, red);
    MG_CK(cudaGetLastError());
    MG_CK(cudaMemcpyAsync(out, red, sizeof(double), cudaMemcpyDeviceToHost, st));
    MG_CK(cudaStreamSynchronize(st));
    ++launches;
    return MG_OK;
  }
  int lincomb(int64_t n, double a, const double* x, double b, const double* y, double* out) {
    k_lincomb<<<grid_of(n), 256, 0, st>>>(n, a, x, b, y, out);
    ++launches;
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
  }
  int csr(const DevCsr& D, const double* x, double* out) {
    k_csr<<<grid_of(D.n), 256, 0, st>>>(D.n, D.ptr, D.idx, D.val, x, out);
    ++launches;
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
  }
  // G = weights of D x (first: identity)
  int weights(const DevCsr& D, const double* x, bool first, double* t, double* g) {
    MG_RC(csr(D, x, t));
    k_max_abs<<<1, kRed, 0, st>>>(D.n, t, red);
    k_weights<<<grid_of(D.n), 256, 0, st>>>(D.n, t, red, first ? 1 : 0, g);
    launches += 2;
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
  }
  // data = L v, v on the cells of `level`
  int apply_L(int level, const double* v, void* data) {
    if (mode == MG_DATA_PROJECTED) {
      MG_RC(mg_jacobian_apply(M, level, eps, shots, wav, dt, nt, v, tr, st, fl));
      return mg_project(u, tr, R, nt, dt, static_cast<double*>(data), st, 0);
    }
    return mg_jacobian_apply(M, level, eps, shots, wav, dt, nt, v, static_cast<float*>(data), st,
                             fl);
  }
  // g = L^T data on the cells of `level`
  int apply_LT(int level, const void* data, double* g) {
    const float* w = static_cast<const float*>(data);
    if (mode == MG_DATA_PROJECTED) {
      MG_RC(mg_projected_weights(u, static_cast<const double*>(data), R, nt, dt, tr2, st, 0));
      w = tr2;
    }
    return mg_jacobian_T_apply(M, level, eps, shots, wav, dt, nt, w, g, P.ckpt_every, st,
                               fl | MG_REUSE_CHECKPOINTS);
  }
  void* data_buf() { return mode == MG_DATA_PROJECTED ? (void*)pd : (void*)tr; }

  // Conjugate gradients on A x = b from x = 0; A symmetric positive definite
  // on the subspace the operator keeps.  Returns iterations and the final
  // relative residual.
  template <class Op>
  int cg(int64_t n, Op&& op, const double* b, double* x, double* r, double* p, double* q,
         int* iters, double* relres) {
    MG_RC(lincomb(n, 0.0, b, 0.0, nullptr, x));
    MG_RC(lincomb(n, 1.0, b, 0.0, nullptr, r));
    MG_RC(lincomb(n, 1.0, b, 0.0, nullptr, p));
    double rr = 0.0, bb = 0.0;
    MG_RC(dot(n, r, r, &rr));
    bb = rr;
    *iters = 0;
    *relres = 0.0;
    if (bb == 0.0) return MG_OK;
    for (int it = 1; it <= P.n_cg; ++it) {
      MG_RC(op(p, q));
      double pq = 0.0;
      MG_RC(dot(n, p, q, &pq));
      if (!(pq > 0.0)) break;  // breakdown: keep the current iterate
      const double a = rr / pq;
      MG_RC(lincomb(n, 1.0, x, a, p, x));
      MG_RC(lincomb(n, 1.0, r, -a, q, r));
      double rr2 = 0.0;
      MG_RC(dot(n, r, r, &rr2));
      *iters = it;
      *relres = std::sqrt(rr2 / bb);
      if (*relres <= P.cg_rtol) break;
      MG_RC(lincomb(n, 1.0, r, rr2 / rr, p, p));
      rr = rr2;
    }
    return MG_OK;
  }
};

}  // namespace
}  // namespace mg

extern "C" int mg_tv_reconstruct_levels(mg_mesh* M, const int* levels, int n_levels,
                                        const double* eps0, const mg_shots* shots,
                                        const double* wavelet, double dt, int nt, int data_mode,
                                        const void* dy, const float* u,
                                        const mg_tv_params* params, double* x_out,
                                        double* history, void* stream, int flags) {
  using namespace mg;
  if (!M || !levels || n_levels < 1 || !eps0 || !shots || !wavelet || !dy || !params ||
      !x_out || nt < 1 || !(dt > 0.0))
    return MG_ERR_ARG;
  if (data_mode != MG_DATA_TRACES && data_mode != MG_DATA_PROJECTED) return MG_ERR_ARG;
  if (data_mode == MG_DATA_PROJECTED && !u) return MG_ERR_ARG;
  if (flags & ~(MG_HOST_PTRS | MG_ALLOW_CFL)) return MG_ERR_UNSUPPORTED;
  const mg_tv_params Pm = *params;
  if (!(Pm.alpha > 0.0) || !(Pm.beta >= 0.0) || Pm.n_outer < 1 || Pm.n_cg < 1 ||
      !(Pm.cg_rtol >= 0.0) || !(Pm.keep_frac > 0.0 && Pm.keep_frac <= 1.0) || Pm.ckpt_every < 1)
    return MG_ERR_ARG;
  const HostMesh* hm = host_mesh(M);
  if (!hm) return MG_ERR_ARG;
  for (int i = 0; i < n_levels; ++i)
    if (levels[i] < 0 || levels[i] >= hm->n_levels || (i > 0 && levels[i] <= levels[i - 1]))
      return MG_ERR_ARG;
  const int level_c = levels[0];
  const int nf = n_levels - 1;  // fine levels f_1 .. f_nf
  int dev_prev = 0;
  if (cudaGetDevice(&dev_prev) != cudaSuccess) return MG_ERR_CUDA;
  if (cudaSetDevice(mesh_device(M)) != cudaSuccess) return MG_ERR_CUDA;
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{dev_prev};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool host = flags & MG_HOST_PTRS;
  const int64_t R = shots->n_shots >= 0 && shots->rec_ptr ? shots->rec_ptr[shots->n_shots] : -1;
  if (R < 0) return MG_ERR_ARG;

  // host-side structure: level graphs, D matrices, one basis per fine level
  Facets F;
  MG_RC(interior_facets(*hm, F));
  const Csr gc = level_graph(*hm, F, level_c);
  const Csr Dc = reg_matrix(gc, Pm.beta);
  const int64_t n_c = hm->n_cells_level[level_c];
  struct Fine {
    int level = 0;
    int64_t n = 0, n_b = 0;
    Csr D;
    Basis B;
    std::vector<int32_t> parent;  // cell of this level -> cell of the previous listed level
    DevCsr dD;
    double *x = nullptr, *g = nullptr, *mask = nullptr, *cells = nullptr, *comp = nullptr;
    int32_t *plus = nullptr, *minus = nullptr, *cfun = nullptr, *parent_d = nullptr;
    int64_t* cptr = nullptr;
    double* csign = nullptr;
  };
  std::vector<Fine> FL(nf);
  int64_t nmax = n_c, nb_max = 0;
  for (int i = 0; i < nf; ++i) {
    Fine& f = FL[i];
    f.level = levels[i + 1];
    const int prev = levels[i];
    const Csr gf = level_graph(*hm, F, f.level);
    f.D = reg_matrix(gf, Pm.beta);
    f.n = hm->n_cells_level[f.level];
    f.parent.assign(f.n, -1);
    for (int64_t e = 0; e < hm->m; ++e)
      f.parent[hm->ancestors[f.level][e]] = hm->ancestors[prev][e];
    MG_RC(fine_basis(gf, f.parent, hm->n_cells_level[prev], f.B));
    f.n_b = (int64_t)f.B.plus.size();
    nmax = std::max(nmax, std::max(f.n, f.n_b));
    nb_max = std::max(nb_max, f.n_b);
  }

  Arena A(st);
  Solver S;
  S.M = M;
  S.shots = shots;
  S.dt = dt;
  S.nt = nt;
  S.mode = data_mode;
  S.P = Pm;
  S.st = st;
  S.fl = flags & MG_ALLOW_CFL;
  S.R = R;
  S.A = &A;
  // inputs on the device
  const int64_t m = hm->m;
  const size_t dlen = data_mode == MG_DATA_PROJECTED ? 2 * (size_t)R : (size_t)R * nt;
  const size_t dbytes = dlen * (data_mode == MG_DATA_PROJECTED ? sizeof(double) : sizeof(float));
  if (host) {
    double *e = nullptr, *w = nullptr;
    void* d = nullptr;
    MG_RC(A.get(&e, m));
    MG_RC(A.get(&w, nt));
    MG_RC(A.get(reinterpret_cast<unsigned char**>(&d), dbytes));
    MG_CK(cudaMemcpyAsync(e, eps0, m * sizeof(double), cudaMemcpyHostToDevice, st));
    MG_CK(cudaMemcpyAsync(w, wavelet, nt * sizeof(double), cudaMemcpyHostToDevice, st));
    MG_CK(cudaMemcpyAsync(d, dy, dbytes, cudaMemcpyHostToDevice, st));
    S.eps = e;
    S.wav = w;
    S.dy = d;
    if (data_mode == MG_DATA_PROJECTED) {
      float* uu = nullptr;
      MG_RC(A.get(&uu, (size_t)R * nt));
      MG_CK(cudaMemcpyAsync(uu, u, (size_t)R * nt * sizeof(float), cudaMemcpyHostToDevice, st));
      S.u = uu;
    }
  } else {
    S.eps = eps0;
    S.wav = wavelet;
    S.dy = dy;
    S.u = u;
  }
  MG_RC(A.get(&S.tr, (size_t)R * nt));
  MG_RC(A.get(&S.tr2, (size_t)R * nt));
  MG_RC(A.get(&S.pd, 2 * (size_t)R));
  MG_RC(A.get(&S.pd2, 2 * (size_t)R));
  MG_RC(A.get(&S.red, 4));
  DevCsr dDc;
  MG_RC(A.put_csr(dDc, Dc));
  // coarse vectors and shared CG scratch
  double *xc, *bc, *r, *p, *q, *t, *gcw, *v1, *v2, *bb = nullptr, *all = nullptr;
  MG_RC(A.get(&xc, n_c));
  MG_RC(A.get(&bc, n_c));
  MG_RC(A.get(&r, nmax));
  MG_RC(A.get(&p, nmax));
  MG_RC(A.get(&q, nmax));
  MG_RC(A.get(&t, nmax));
  MG_RC(A.get(&gcw, n_c));
  MG_RC(A.get(&v1, nmax));
  MG_RC(A.get(&v2, nmax));
  if (nf > 0) {
    MG_RC(A.get(&bb, nb_max));
    MG_RC(A.put(&all, std::vector<double>(nb_max, 1.0)));  // a mask of ones
  }
  for (Fine& f : FL) {
    MG_RC(A.put_csr(f.dD, f.D));
    MG_RC(A.get(&f.x, f.n_b));
    MG_RC(A.get(&f.g, f.n));
    MG_RC(A.get(&f.mask, f.n_b));
    MG_RC(A.get(&f.cells, f.n));
    MG_RC(A.get(&f.comp, f.n));
    MG_RC(A.put(&f.plus, f.B.plus));
    MG_RC(A.put(&f.minus, f.B.minus));
    MG_RC(A.put(&f.cptr, f.B.cptr));
    MG_RC(A.put(&f.cfun, f.B.cfun));
    MG_RC(A.put(&f.csign, f.B.csign));
    MG_RC(A.put(&f.parent_d, f.parent));
    MG_CK(cudaMemsetAsync(f.x, 0, f.n_b * sizeof(double), st));
  }
  MG_CK(cudaMemsetAsync(xc, 0, n_c * sizeof(double), st));

  // one forward with checkpoints; every J^T reuses them
  MG_RC(mg_forward(M, S.eps, shots, S.wav, dt, nt, S.tr, Pm.ckpt_every, st,
                   S.fl | MG_KEEP_CHECKPOINTS));
  // b_c = L_c^T dy (the same on every outer step)
  MG_RC(S.apply_LT(level_c, S.dy, bc));

  const double alpha = Pm.alpha;
  // A_c p = L_c^T L_c p + alpha D_c G_c D_c p
  auto op_c = [&](const double* pin, double* out) -> int {
    MG_RC(S.apply_L(level_c, pin, S.data_buf()));
    MG_RC(S.apply_LT(level_c, S.data_buf(), out));
    MG_RC(S.csr(dDc, pin, v1));
    k_mul<<<grid_of(n_c), 256, 0, st>>>(n_c, gcw, v1);
    MG_CK(cudaGetLastError());
    MG_RC(S.csr(dDc, v1, v2));
    return S.lincomb(n_c, 1.0, out, alpha, v2, out);
  };
  // A_fi p = mask R_fi^T (L^T L + alpha D_li G_fi D_li) R_fi mask p   (level l_i cells)
  const Fine* cur = nullptr;
  auto op_f = [&](const double* pin, double* out) -> int {
    const Fine& f = *cur;
    k_rf<<<grid_of(f.n), 256, 0, st>>>(f.n, f.cptr, f.cfun, f.csign, f.mask, pin, f.cells);
    MG_CK(cudaGetLastError());
    MG_RC(S.apply_L(f.level, f.cells, S.data_buf()));
    MG_RC(S.apply_LT(f.level, S.data_buf(), v1));
    MG_RC(S.csr(f.dD, f.cells, v2));
    k_mul<<<grid_of(f.n), 256, 0, st>>>(f.n, f.g, v2);
    MG_CK(cudaGetLastError());
    MG_RC(S.csr(f.dD, v2, t));
    MG_RC(S.lincomb(f.n, 1.0, v1, alpha, t, v1));
    k_rft<<<grid_of(f.n_b), 256, 0, st>>>(f.n_b, f.plus, f.minus, f.mask, v1, out);
    S.launches += 2;
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
  };

  const int hw = 2 * n_levels;  // history entries per outer step
  std::vector<double> hist((size_t)hw * Pm.n_outer, 0.0);
  std::vector<double> prev_h, mask_h;
  for (int l = 0; l < Pm.n_outer; ++l) {
    // (2) coarse update
    MG_RC(S.weights(dDc, xc, l == 0, t, gcw));
    int it = 0;
    double rel = 0.0;
    MG_RC(S.cg(n_c, op_c, bc, xc, r, p, q, &it, &rel));
    hist[(size_t)hw * l + 0] = it;
    hist[(size_t)hw * l + 1] = rel;
    // (3) and the recursion over f_1 .. f_nf: comp is the reconstruction
    // assembled so far, on the cells of the previous listed level
    const double* comp = xc;
    int64_t n_prev = n_c;
    int level_prev = level_c;
    for (int i = 0; i < nf; ++i) {
      Fine& f = FL[i];
      cur = &f;
      // compression: basis functions under the top keep_frac of the
      // previous level's cells by |comp|
      prev_h.resize(n_prev);
      MG_CK(cudaMemcpyAsync(prev_h.data(), comp, n_prev * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
      MG_CK(cudaStreamSynchronize(st));
      std::vector<int64_t> order(n_prev);
      std::iota(order.begin(), order.end(), 0);
      std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        return std::fabs(prev_h[a]) > std::fabs(prev_h[b]);
      });
      const int64_t keep = std::min<int64_t>(
          n_prev, (int64_t)std::ceil(Pm.keep_frac * (double)n_prev - 1e-12));
      std::vector<char> kept(n_prev, 0);
      for (int64_t k = 0; k < keep; ++k) kept[order[k]] = 1;
      mask_h.resize(f.n_b);
      for (int64_t k = 0; k < f.n_b; ++k) mask_h[k] = kept[f.B.coarse[k]] ? 1.0 : 0.0;
      MG_CK(cudaMemcpyAsync(f.mask, mask_h.data(), f.n_b * sizeof(double),
                            cudaMemcpyHostToDevice, st));
      // G_fi from the previous outer step's coordinates (zero outside its
      // kept set): cells = R_fi x_fi
      k_rf<<<grid_of(f.n), 256, 0, st>>>(f.n, f.cptr, f.cfun, f.csign, all, f.x, f.cells);
      MG_CK(cudaGetLastError());
      MG_RC(S.weights(f.dD, f.cells, l == 0, t, f.g));
      // residual data r = dy - L comp (= dy - L_c x_c - sum_k<i L_fk x_fk),
      // then b = mask R_fi^T L_fi^T r
      MG_RC(S.apply_L(level_prev, comp, S.data_buf()));
      void* rd;
      if (data_mode == MG_DATA_PROJECTED) {
        k_sub_d<<<grid_of(2 * R), 256, 0, st>>>(2 * R, static_cast<const double*>(S.dy), S.pd,
                                                 S.pd2);
        rd = S.pd2;
      } else {
        k_sub_f<<<grid_of(R * nt), 256, 0, st>>>(R * nt, static_cast<const float*>(S.dy), S.tr,
                                                  S.tr2);
        rd = S.tr2;
      }
      MG_CK(cudaGetLastError());
      if (data_mode == MG_DATA_PROJECTED) {
        MG_RC(S.apply_LT(f.level, rd, v1));
      } else {
        // apply_LT reads its traces directly (tr2 holds r)
        MG_RC(mg_jacobian_T_apply(M, f.level, S.eps, shots, S.wav, dt, nt, S.tr2, v1,
                                  Pm.ckpt_every, st, S.fl | MG_REUSE_CHECKPOINTS));
      }
      k_rft<<<grid_of(f.n_b), 256, 0, st>>>(f.n_b, f.plus, f.minus, f.mask, v1, bb);
      MG_CK(cudaGetLastError());
      MG_RC(S.cg(f.n_b, op_f, bb, f.x, r, p, q, &it, &rel));
      hist[(size_t)hw * l + 2 * (i + 1)] = it;
      hist[(size_t)hw * l + 2 * (i + 1) + 1] = rel;
      // comp on this level: the previous level's value plus R_fi x_fi
      k_rf<<<grid_of(f.n), 256, 0, st>>>(f.n, f.cptr, f.cfun, f.csign, all, f.x, f.cells);
      k_level_sum<<<grid_of(f.n), 256, 0, st>>>(f.n, f.parent_d, comp, f.cells, f.comp);
      MG_CK(cudaGetLastError());
      S.launches += 2;
      comp = f.comp;
      n_prev = f.n;
      level_prev = f.level;
    }
  }
  // (4) x = R_c x_c + sum_i R_fi x_fi on the last level
  const int64_t n_out = nf ? FL[nf - 1].n : n_c;
  const double* xl = nf ? FL[nf - 1].comp : xc;
  if (host) {
    MG_CK(cudaMemcpyAsync(x_out, xl, n_out * sizeof(double), cudaMemcpyDeviceToHost, st));
  } else {
    MG_CK(cudaMemcpyAsync(x_out, xl, n_out * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  if (history) std::memcpy(history, hist.data(), hist.size() * sizeof(double));
  add_launches(M, S.launches);
  MG_CK(cudaStreamSynchronize(st));
  return MG_OK;
}

extern "C" int mg_tv_reconstruct(mg_mesh* M, int level_c, int level_f, const double* eps0,
                                 const mg_shots* shots, const double* wavelet, double dt, int nt,
                                 int data_mode, const void* dy, const float* u,
                                 const mg_tv_params* params, double* x_out, double* history,
                                 void* stream, int flags) {
  const int levels[2] = {level_c, level_f};
  const int n = level_f >= 0 ? 2 : 1;
  if (!params || params->n_outer < 1) return MG_ERR_ARG;
  std::vector<double> h((size_t)2 * n * params->n_outer, 0.0);
  const int rc = mg_tv_reconstruct_levels(M, levels, n, eps0, shots, wavelet, dt, nt, data_mode,
                                          dy, u, params, x_out, history ? h.data() : nullptr,
                                          stream, flags);
  if (rc == MG_OK && history) {
    for (int l = 0; l < params->n_outer; ++l)
      for (int k = 0; k < 4; ++k) history[4 * l + k] = k < 2 * n ? h[(size_t)2 * n * l + k] : 0.0;
  }
  return rc;
}
