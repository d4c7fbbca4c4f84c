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
  functions of the top third of the coarse cells.
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
