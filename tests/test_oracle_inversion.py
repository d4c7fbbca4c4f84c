"""Pins of the reconstruction oracle (Sec. II: reconstruction procedure,
coarse-to-fine approach, compression of coefficients).

Facts that do not come from the oracle:
* shared-boundary measures on the uniform right-triangle grid: a square's
  diagonal h*sqrt(2) inside it, legs h between squares, and the full
  perimeter h (2 + sqrt 2) for every interior triangle;
* D 1 = beta 1, symmetry, and the kernel of D (beta = 0) being the constants
  of a connected level;
* the 2D fluctuation pairs join the centre child (whose centroid is the
  parent's centroid) to each corner child; in 2D and 3D the coarse and fine
  coordinates together form a basis of the fine cell space (the
  decomposition is unique);
* the first iterate solves the Tikhonov problem (its objective has zero
  directional derivatives, by finite differences); later iterates never
  increase ||Lx - dy||^2 + 2 alpha ||Dx||_1 (majorise-minimise) and the last
  one is not improved by random perturbations;
* data that a coarse vector explains exactly is recovered by the coarse step
  with a vanishing fine correction; the compression keeps the basis
  functions of the top third of the coarse cells;
* with more than two levels and L = I on a uniformly refined mesh (every
  cell of a level has the same number of last-level descendants, so the
  coarse space and the fluctuation spaces are mutually orthogonal), the
  recursion is the multiresolution split of the data: the coarse step gives
  the level-0 means, the first correction the level-1 means minus the
  level-0 means, the last the data minus the level-1 means, each only under
  the cells the compression keeps;
* with a general L and vanishing alpha every step is the least-squares fit
  of the data left by the coarser steps: the data residual of the
  reconstruction assembled up to level i is orthogonal to the kept columns
  of L_fi (for i = 0, to the columns of L_c);
* with two levels the recursion is the two-level procedure.
"""
import math

import numpy as np
import pytest

from oracle import inversion as inv
from oracle import wave
from workloads import configs, meshes


def _level_data(m, level):
    anc = m.ancestor(level)
    return anc, inv.shared_measure(m.coords, m.cells, anc, m.n_cells[level])


def test_shared_measure_closed_form_on_uniform_grid():
    m = meshes.square_mesh(4, 1)          # level 0: 4x4 squares of side h = 0.5
    h = 0.5
    anc, s = _level_data(m, 0)
    vals = np.unique(np.round(s[s > 0], 12))
    assert np.allclose(vals, sorted([h, h * math.sqrt(2)]), rtol=1e-12)
    # interior triangles: boundary entirely shared, perimeter h (2 + sqrt 2)
    n0 = m.n_cells[0]
    cent = np.array([m.coords[m.cells[anc == c]].reshape(-1, 2).mean(0) for c in range(n0)])
    interior = np.all(np.abs(cent) < 1 - h, axis=1)
    assert interior.sum() > 0
    assert np.allclose(s[interior].sum(1), h * (2 + math.sqrt(2)), rtol=1e-12)
    assert np.array_equal(s, s.T)


def test_regularisation_matrix_properties():
    m = meshes.square_mesh(4, 1)
    _, s = _level_data(m, 0)
    for beta in (0.0, 0.3):
        D = inv.regularisation_matrix(s, beta)
        assert np.allclose(D, D.T)
        assert np.allclose(D @ np.ones(len(D)), beta, atol=1e-13)
    D = inv.regularisation_matrix(s, 0.0)
    off = -D[~np.eye(len(D), dtype=bool)]
    assert np.allclose(np.unique(np.round(off[off > 0], 12)), [1 / math.sqrt(2), 1.0])
    ev = np.linalg.eigvalsh(D)
    assert ev.min() > -1e-12 and np.sum(np.abs(ev) < 1e-10) == 1   # kernel = constants


def test_fine_basis_2d_is_centre_corner_pairs():
    m = meshes.square_mesh(2, 2)
    anc_f, s_f = _level_data(m, 2)
    parent = inv.parent_map(m.cell_parent, m.n_cells, 1, 2)
    basis, Rc, Rf = inv.fine_basis(s_f, parent, m.n_cells[1])
    assert len(basis) == 3 * m.n_cells[1]
    anc_c = m.ancestor(1)
    for p, q, c in basis:
        # the minus cell is the centre child: its centroid is the parent's
        cq = m.coords[m.cells[q]].mean(0)
        pts = np.unique(np.round(m.coords[m.cells[anc_c == c]].reshape(-1, 2), 12), axis=0)
        # the parent's three corners are the children's vertices farthest from it
        corners = pts[np.argsort(np.linalg.norm(pts - cq, axis=1))[-3:]]
        assert np.allclose(cq, corners.mean(0), atol=1e-12)
        assert s_f[p, q] > 0 and parent[p] == c and parent[q] == c
    B = np.hstack([Rc, Rf])
    assert B.shape[0] == B.shape[1] and np.linalg.matrix_rank(B) == B.shape[0]


def test_fine_basis_3d_spans_the_fine_space():
    w = configs.tiny_3d()
    m = w.mesh
    anc_f, s_f = _level_data(m, 1)
    parent = inv.parent_map(m.cell_parent, m.n_cells, 0, 1)
    basis, Rc, Rf = inv.fine_basis(s_f, parent, m.n_cells[0])
    assert len(basis) == 7 * m.n_cells[0]
    assert all(s_f[p, q] > 0 for p, q, _ in basis)
    B = np.hstack([Rc, Rf])
    assert np.linalg.matrix_rank(B) == B.shape[0] == B.shape[1]


@pytest.fixture(scope="module")
def lin():
    """Dense trace Jacobian of tiny_2d w.r.t. its level-1 cells (32 columns)."""
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=90)
    m, sh = w.mesh, w.shots
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    anc1 = m.ancestor(1)
    cols = []
    for c in range(m.n_cells[1]):
        e = np.zeros(m.n_cells[1])
        e[c] = 1.0
        cols.append(wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec,
                                 wave.prolong(e, anc1)).ravel())
    L1 = np.stack(cols, 1)
    _, s1 = _level_data(m, 1)
    return w, L1, s1


def test_first_iterate_is_tikhonov_and_objective_decreases(lin):
    w, L, s1 = lin
    D = inv.regularisation_matrix(s1, 0.05)
    rng = np.random.default_rng(0)
    x_true = np.where(np.arange(L.shape[1]) % 5 == 0, 1.0, 0.0)
    dy = L @ x_true + 0.01 * np.abs(L @ x_true).max() * rng.standard_normal(L.shape[0])
    alpha = 1e-3 * np.linalg.norm(L, 2) ** 2
    xs = inv.tv_irls(L, D, dy, alpha, 60)
    tik = lambda x: float(np.sum((L @ x - dy) ** 2) + alpha * np.sum((D @ x) ** 2))
    h = 1e-4 * np.linalg.norm(xs[0])
    for _ in range(5):
        d = rng.standard_normal(L.shape[1])
        d /= np.linalg.norm(d)
        slope = (tik(xs[0] + h * d) - tik(xs[0] - h * d)) / (2 * h)
        assert abs(slope) <= 1e-6 * tik(xs[0]) / np.linalg.norm(xs[0])
    F = [inv.objective(L, D, dy, x, alpha) for x in xs]
    assert all(F[i + 1] <= F[i] * (1 + 1e-10) for i in range(len(F) - 1))
    assert F[-1] < F[0]
    for _ in range(20):
        d = rng.standard_normal(L.shape[1])
        assert inv.objective(L, D, dy, xs[-1] + 1e-3 * np.linalg.norm(xs[-1]) * d /
                             np.linalg.norm(d), alpha) >= F[-1] * (1 - 1e-6)


def test_coarse_to_fine_recovers_coarse_explained_data(lin):
    w, L1, s1 = lin
    m = w.mesh
    _, s0 = _level_data(m, 0)
    parent = inv.parent_map(m.cell_parent, m.n_cells, 0, 1)
    basis, Rc, Rf = inv.fine_basis(s1, parent, m.n_cells[0])
    xc_true = np.linspace(-1.0, 2.0, m.n_cells[0])
    dy = L1 @ Rc @ xc_true
    out = inv.coarse_to_fine(L1, inv.regularisation_matrix(s1, 0.1),
                             inv.regularisation_matrix(s0, 0.1), Rc, Rf, basis, dy,
                             alpha=1e-12 * np.linalg.norm(L1 @ Rc, 2) ** 2, n_outer=2)
    xc, xb, x, K = out[0]
    assert np.linalg.norm(xc - xc_true) <= 1e-5 * np.linalg.norm(xc_true)
    assert np.linalg.norm(Rf @ xb) <= 1e-5 * np.linalg.norm(Rc @ xc)
    # compression: the basis functions of the top third of the coarse cells
    k = math.ceil(m.n_cells[0] / 3)
    top = set(np.argsort(-np.abs(xc), kind="stable")[:k])
    assert sorted(K) == [i for i, (_, _, c) in enumerate(basis) if c in top]
    assert len(K) == 3 * k


def _means(v_top, P):
    """Mean of last-level values over the descendants of each level cell."""
    return (P.T @ v_top) / P.sum(axis=0)


def _top(values, k):
    """Indices of the k largest |values| (ties: lower index first)."""
    return np.argsort(-np.abs(values), kind="stable")[:k]


@pytest.mark.parametrize("make", [lambda: meshes.square_mesh(2, 2),
                                  lambda: meshes.ellipsoid_mesh(2, (2, 2, 2))],
                         ids=["square_2d", "ellipsoid_3d"])
@pytest.mark.parametrize("keep", [1.0, 1.0 / 3.0])
def test_levels_recursion_with_identity_data_is_the_multiresolution_split(make, keep):
    m = make()
    Ds, Ps, bases, Rs = inv.hierarchy(m.coords, m.cells, m.cell_parent, m.n_cells, [0, 1, 2],
                                      0.5)
    n = m.n_cells[2]
    assert Ps[0].shape[1] + sum(R.shape[1] for R in Rs[1:]) == n
    dy = np.random.default_rng(3).standard_normal(n)
    xc, xfs, x, Ks = inv.coarse_to_fine_levels(np.eye(n), Ds, Ps, bases, Rs, dy, alpha=1e-12,
                                               n_outer=1, keep_frac=keep)[0]
    m0, m1 = _means(dy, Ps[0]), _means(dy, Ps[1])
    assert np.allclose(xc, m0, rtol=0, atol=1e-9)
    k1 = _top(m0, math.ceil(keep * m.n_cells[0] - 1e-12))
    on1 = np.isin(inv.parent_map(m.cell_parent, m.n_cells, 0, 2), k1)
    x1 = Ps[0] @ m0 + on1 * (Ps[1] @ m1 - Ps[0] @ m0)
    k2 = _top(_means(x1, Ps[1]), math.ceil(keep * m.n_cells[1] - 1e-12))
    on2 = np.isin(inv.parent_map(m.cell_parent, m.n_cells, 1, 2), k2)
    expect = x1 + on2 * (dy - Ps[1] @ m1)
    assert np.linalg.norm(x - expect) <= 1e-8 * np.linalg.norm(dy)
    if keep == 1.0:
        assert np.linalg.norm(x - dy) <= 1e-8 * np.linalg.norm(dy)
    else:
        assert 0 < len(Ks[1]) < Rs[2].shape[1]


def test_levels_recursion_with_two_levels_is_coarse_to_fine(lin):
    w, L1, s1 = lin
    m = w.mesh
    _, s0 = _level_data(m, 0)
    parent = inv.parent_map(m.cell_parent, m.n_cells, 0, 1)
    basis, Rc, Rf = inv.fine_basis(s1, parent, m.n_cells[0])
    rng = np.random.default_rng(4)
    dy = L1 @ rng.standard_normal(m.n_cells[1])
    alpha = 1e-3 * np.linalg.norm(L1 @ Rc, 2) ** 2
    a = inv.coarse_to_fine(L1, inv.regularisation_matrix(s1, 0.2),
                           inv.regularisation_matrix(s0, 0.2), Rc, Rf, basis, dy, alpha, 3)
    Ds, Ps, bases, Rs = inv.hierarchy(m.coords, m.cells, m.cell_parent, m.n_cells, [0, 1], 0.2)
    b = inv.coarse_to_fine_levels(L1, Ds, Ps, bases, Rs, dy, alpha, 3)
    for (xc, xb, x, K), (yc, yfs, y, Ks) in zip(a, b):
        assert K == Ks[0]
        assert np.linalg.norm(xc - yc) <= 1e-10 * np.linalg.norm(xc)
        assert np.linalg.norm(xb - yfs[0]) <= 1e-10 * np.linalg.norm(xb)
        assert np.linalg.norm(x - y) <= 1e-10 * np.linalg.norm(x)


def test_levels_recursion_fits_what_the_coarser_levels_left():
    m = meshes.square_mesh(2, 2)
    Ds, Ps, bases, Rs = inv.hierarchy(m.coords, m.cells, m.cell_parent, m.n_cells, [0, 1, 2],
                                      0.5)
    rng = np.random.default_rng(6)
    L = rng.standard_normal((300, m.n_cells[2]))
    dy = rng.standard_normal(300)
    xc, xfs, x, Ks = inv.coarse_to_fine_levels(L, Ds, Ps, bases, Rs, dy,
                                               alpha=1e-12 * np.linalg.norm(L, 2) ** 2,
                                               n_outer=1)[0]
    scale = np.linalg.norm(L, 2) * np.linalg.norm(dy)
    x_top = Ps[0] @ xc
    assert np.linalg.norm((L @ Ps[0]).T @ (dy - L @ x_top)) <= 1e-8 * scale
    for i in (1, 2):
        x_top = x_top + Ps[i] @ (Rs[i] @ xfs[i - 1])
        cols = (L @ Ps[i] @ Rs[i])[:, Ks[i - 1]]
        assert len(Ks[i - 1]) > 0
        assert np.linalg.norm(cols.T @ (dy - L @ x_top)) <= 1e-8 * scale
    assert np.allclose(x_top, x, rtol=0, atol=1e-12 * np.abs(x).max())
