"""Oracle: the TV-regularised reconstruction of Sec. II (reconstruction
procedure, coarse-to-fine approach, compression of coefficients), dense FP64
on tiny problems.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module.

The linearised model y - y0 = L (x - x0) + n, with L the Jacobian of the data
with respect to the cell values x of a nested level (x0 = 0: x is the
perturbation of the background permittivity), is inverted by the iteration
(tv_iteration)

    x_{l+1} = x0 + (L^T L + alpha D^T G_l D)^{-1} L^T (y - y0),
    G_0 = I,  G_l = diag(|D (x_l - x0)|)^{-1},

with the regularisation matrix (d_mat) over the cells of the level.  Here
every linear system is solved directly (numpy.linalg.solve) from a dense L
built column by column; the CUDA driver uses matrix-free conjugate
gradients, so the two share no solver.

Readings of the passages that the paper leaves open (also listed in the
design notes):
* (d_mat): D_ij = -s_ij / s_max for i != j, with s_ij the measure of the
  boundary shared by cells i and j; D_ii = beta + sum_{j != i} s_ij / s_max
  (the i = j integral read as the part of the cell's boundary shared with
  other cells), so D 1 = beta 1 and (D x)_i = beta x_i + sum_j s_ij (x_i -
  x_j) / s_max penalises jumps over the edges.  D is symmetric; the
  iteration is written with D^T G D, which is D G D.
* G_l: entries |D(x_l - x0)|_i below tau = 1e-8 max_i |D(x_l - x0)|_i are
  raised to tau (the inverse is otherwise unbounded); G = I while D(x_l -
  x0) = 0.
* The iteration is a majorise-minimise step of
  F(x) = ||L(x - x0) - (y - y0)||^2 + 2 alpha ||D(x - x0)||_1, so F does not
  increase; the paper writes the weight of the 1-norm as 2 sqrt(alpha), which
  would correspond to sqrt(alpha) D^T G D in the iteration.  The iteration
  is implemented as printed.
* Coarse-to-fine (two nested levels c < f, steps (1)-(5)): R_c maps a level-c
  vector to level f (each fine cell takes its parent's value); R_f maps the
  coordinates of the fine fluctuations.  Basis of the fluctuations inside a
  coarse cell: +1 on one child, -1 on an adjacent child (sharing a facet),
  along a breadth-first spanning tree of the children's facet adjacency
  rooted at the child with the most neighbours among its siblings (ties: the
  lowest index); siblings are visited in index order.  In 2D the root is the
  centre child, adjacent to the three corners: the pairs of Sec. II.
  L_c = L R_c, L_f = L R_f, D_c = D of level c, D_f = D_level_f R_f (so
  D_f^T G D_f, G over the level-f cells).  Every step starts from x0 = 0.
* Compression: the kept fine basis functions are those of the
  ceil(keep_frac n_c) coarse cells with the largest |x^(c)_{l+1} - x^(c)_0|
  (ties: lower index), keep_frac = 1/3 in the paper; x^(f) is zero outside
  the kept set, and G for the fine step is formed from the full x^(f)_l.
* More than two nested levels l_0 < l_1 < ... < l_nf (tv_iteration_3): L is
  the Jacobian on the cells of the last level; f_i is the fluctuation space
  of level l_i inside the cells of level l_{i-1} (the basis above), with
  L_fi = L P_i R_fi (P_i prolongs level l_i to the last level) and
  D_fi = D_level_li R_fi.  The printed residual sums L_{f_i} x^(f_i) over
  k = 1..i-1, which refers to the unknown itself; it is read as
  sum_k L_{f_k} [x^(f_k)_{l+1} - x^(f_k)_0], the corrections of the coarser
  fine levels found in the same outer step.  Compression at level i ranks
  the cells of level l_{i-1} by |x| of the reconstruction assembled so far
  (coarse plus the corrections of levels 1..i-1), which for i = 1 is
  |x^(c)|.  With two levels this is steps (1)-(5).
"""
from __future__ import annotations

import math

import numpy as np

from . import fem


def parent_map(cell_parent, n_cells, level_c: int, level_f: int) -> np.ndarray:
    """Level-c ancestor of every level-f cell (level_c <= level_f)."""
    anc = np.arange(n_cells[level_f], dtype=np.int64)
    for l in range(level_f, level_c, -1):
        anc = np.asarray(cell_parent[l - 1], dtype=np.int64)[anc]
    return anc


def shared_measure(coords, cells, ancestor, n_level: int) -> np.ndarray:
    """s[a][b]: total measure of the finest facets between a descendant of
    level cell a and a descendant of level cell b (a != b); dense."""
    d = coords.shape[1]
    owners = {}
    for e in range(cells.shape[0]):
        for k in range(d + 1):
            f = tuple(sorted(int(v) for v in np.delete(cells[e], k)))
            owners.setdefault(f, []).append(e)
    s = np.zeros((n_level, n_level))
    for f, es in owners.items():
        if len(es) != 2:
            continue
        a, b = int(ancestor[es[0]]), int(ancestor[es[1]])
        if a != b:
            mu = fem.facet_measure(coords, np.array([f]))[0]
            s[a, b] += mu
            s[b, a] += mu
    return s


def regularisation_matrix(s: np.ndarray, beta: float) -> np.ndarray:
    """D of (d_mat) from the shared-boundary measures s (reading above)."""
    smax = s.max()
    D = -s / smax
    D[np.diag_indices_from(D)] = beta + s.sum(axis=1) / smax
    return D


def fine_basis(s_f: np.ndarray, parent: np.ndarray, n_c: int):
    """Fine-fluctuation basis: list of (plus cell, minus cell, coarse cell)
    and the matrices R_c [n_f][n_c], R_f [n_f][n_basis]."""
    n_f = parent.shape[0]
    basis = []
    for c in range(n_c):
        kids = [int(e) for e in np.nonzero(parent == c)[0]]
        degree = [sum(1 for b in kids if b != a and s_f[a, b] > 0) for a in kids]
        root = kids[int(np.argmax(degree))]
        seen = {root}
        queue = [root]
        for a in queue:
            for b in kids:
                if b not in seen and s_f[a, b] > 0:
                    basis.append((b, a, c))
                    seen.add(b)
                    queue.append(b)
        if len(seen) != len(kids):
            raise ValueError("children of a coarse cell are not facet-connected")
    Rc = np.zeros((n_f, n_c))
    Rc[np.arange(n_f), parent] = 1.0
    Rf = np.zeros((n_f, len(basis)))
    for k, (p, m, _) in enumerate(basis):
        Rf[p, k] = 1.0
        Rf[m, k] = -1.0
    return basis, Rc, Rf


def weights(t: np.ndarray, first: bool) -> np.ndarray:
    """Diagonal of G: ones on the first step or while t = 0, else 1/|t|
    with |t| raised to 1e-8 max|t|."""
    a = np.abs(t)
    if first or a.max() == 0.0:
        return np.ones_like(a)
    return 1.0 / np.maximum(a, 1e-8 * a.max())


def objective(L, D, dy, x, alpha) -> float:
    """||L x - dy||^2 + 2 alpha ||D x||_1 (x0 = 0)."""
    r = L @ x - dy
    return float(r @ r + 2.0 * alpha * np.abs(D @ x).sum())


def tv_irls(L, D, dy, alpha: float, n_iter: int):
    """Single-level iteration (tv_iteration) from x0 = 0; the iterates."""
    x = np.zeros(L.shape[1])
    out = []
    for l in range(n_iter):
        g = weights(D @ x, l == 0)
        A = L.T @ L + alpha * D.T @ (g[:, None] * D)
        x = np.linalg.solve(A, L.T @ dy)
        out.append(x.copy())
    return out


def kept_basis(xc: np.ndarray, basis, keep_frac: float):
    """Indices of the fine basis functions kept by the compression."""
    n_c = xc.shape[0]
    k = int(math.ceil(keep_frac * n_c - 1e-12))
    order = sorted(range(n_c), key=lambda c: (-abs(xc[c]), c))
    keep = set(order[:k])
    return [i for i, (_, _, c) in enumerate(basis) if c in keep]


def coarse_to_fine(L_f, D_level_f, D_c, Rc, Rf, basis, dy, alpha: float, n_outer: int,
                   keep_frac: float = 1.0 / 3.0):
    """Steps (1)-(5) with two levels: per outer step the coarse update
    (tv_iteration_0), the compressed fine correction (tv_iteration_2) and
    their sum.  L_f: data x level-f cells.  Returns per step
    (x_c, x_fluct, x_level_f, kept)."""
    Lc = L_f @ Rc
    Lb = L_f @ Rf
    Df = D_level_f @ Rf
    xc = np.zeros(Rc.shape[1])
    xb = np.zeros(Rf.shape[1])
    out = []
    for l in range(n_outer):
        gc = weights(D_c @ xc, l == 0)
        xc = np.linalg.solve(Lc.T @ Lc + alpha * D_c.T @ (gc[:, None] * D_c), Lc.T @ dy)
        K = kept_basis(xc, basis, keep_frac)
        gf = weights(Df @ xb, l == 0)
        r = dy - Lc @ xc
        LK, DK = Lb[:, K], Df[:, K]
        xK = np.linalg.solve(LK.T @ LK + alpha * DK.T @ (gf[:, None] * DK), LK.T @ r)
        xb = np.zeros(Rf.shape[1])
        xb[K] = xK
        out.append((xc.copy(), xb.copy(), Rc @ xc + Rf @ xb, K))
    return out


def hierarchy(coords, cells, cell_parent, n_cells, levels, beta: float):
    """Per listed level l_i (increasing): D of the level, P_i [n_top][n_li]
    (each last-level cell takes its level-l_i ancestor's value) and, for
    i >= 1, the fine_basis of level l_i inside level l_{i-1} with its
    R_fi [n_li][nb_i].  Entry 0 of the basis lists is None."""
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells)
    finest = len(n_cells) - 1
    top = levels[-1]
    Ds, Ps, bases, Rs = [], [], [None], [None]
    for i, lev in enumerate(levels):
        anc = parent_map(cell_parent, n_cells, lev, finest)
        s = shared_measure(coords, cells, anc, n_cells[lev])
        Ds.append(regularisation_matrix(s, beta))
        up = parent_map(cell_parent, n_cells, lev, top)
        P = np.zeros((n_cells[top], n_cells[lev]))
        P[np.arange(n_cells[top]), up] = 1.0
        Ps.append(P)
        if i > 0:
            parent = parent_map(cell_parent, n_cells, levels[i - 1], lev)
            basis, _, Rf = fine_basis(s, parent, n_cells[levels[i - 1]])
            bases.append(basis)
            Rs.append(Rf)
    return Ds, Ps, bases, Rs


def coarse_to_fine_levels(L, Ds, Ps, bases, Rs, dy, alpha: float, n_outer: int,
                          keep_frac: float = 1.0 / 3.0):
    """Steps (1)-(5) with the recursion (tv_iteration_3) over the levels of
    ``hierarchy``; L: data x last-level cells.  Per outer step the coarse
    update (tv_iteration_0), then for i = 1..nf the compressed correction in
    f_i against the data left by the coarse step and by the corrections of
    f_1..f_{i-1} of the same step.  Returns per step
    (x_c, [x_f1, ..], x_last_level, [K_1, ..])."""
    nf = len(Ds) - 1
    Lc = L @ Ps[0]
    Lf = [None] + [L @ Ps[i] @ Rs[i] for i in range(1, nf + 1)]
    Df = [None] + [Ds[i] @ Rs[i] for i in range(1, nf + 1)]
    xc = np.zeros(Ps[0].shape[1])
    xf = [None] + [np.zeros(Rs[i].shape[1]) for i in range(1, nf + 1)]
    out = []
    for l in range(n_outer):
        gc = weights(Ds[0] @ xc, l == 0)
        xc = np.linalg.solve(Lc.T @ Lc + alpha * Ds[0].T @ (gc[:, None] * Ds[0]), Lc.T @ dy)
        new = [None] * (nf + 1)
        kept = []
        for i in range(1, nf + 1):
            # reconstruction so far, on the last level, then on level l_{i-1}
            x_top = Ps[0] @ xc
            for k in range(1, i):
                x_top = x_top + Ps[k] @ (Rs[k] @ new[k])
            prev = (Ps[i - 1].T @ x_top) / Ps[i - 1].sum(axis=0)
            K = kept_basis(prev, bases[i], keep_frac)
            r = dy - Lc @ xc
            for k in range(1, i):
                r = r - Lf[k] @ new[k]
            g = weights(Df[i] @ xf[i], l == 0)
            LK, DK = Lf[i][:, K], Df[i][:, K]
            xK = np.linalg.solve(LK.T @ LK + alpha * DK.T @ (g[:, None] * DK), LK.T @ r)
            new[i] = np.zeros(Rs[i].shape[1])
            new[i][K] = xK
            kept.append(K)
        xf = new
        x = Ps[0] @ xc
        for i in range(1, nf + 1):
            x = x + Ps[i] @ (Rs[i] @ xf[i])
        out.append((xc.copy(), [v.copy() for v in xf[1:]], x, kept))
    return out
