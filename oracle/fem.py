"""Oracle: P1 finite-element matrices of the scalar wave problem, FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module; it exists so that tests, the smoke check and the CPU baseline of the
benchmark can compare the CUDA library against a plain definition.

Definitions (App. A, "Numerical solution of the wave equation"):
* nodal P1 basis phi_j and elementwise P0 flux; eliminating the flux q from
  Eqs. (leap-frog1)-(leap-frog2) leaves sum_k B^(k)T A^-1 B^(k) = K, the P1
  stiffness K_ij = sum_e |e| grad(phi_i).grad(phi_j)  (A_ii = |T_i|,
  B^(k)_ij = int_{T_i} e_k . grad(phi_j)).
* C_ij = int eps phi_i phi_j, here lumped: m_i = sum_{e contains i} eps_e |e|/(d+1).
* First-order absorbing boundary (the boundary law du/dn = -sqrt(eps) du/dt,
  which replaces the paper's split-field PML): lumped boundary matrix
  D_ii = sum_{boundary facets F contains i} sqrt(eps_{e(F)}) |F| / d.

All routines accept complex eps so that complex-step derivatives can be
taken through them.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def simplex_geometry(coords: np.ndarray, cells: np.ndarray):
    """Per cell: measure |e| (float64 [m]) and the gradients of the d+1
    barycentric basis functions (float64 [m, d+1, d])."""
    x = coords[cells]                       # [m, d+1, d]
    d = coords.shape[1]
    E = np.transpose(x[:, 1:, :] - x[:, :1, :], (0, 2, 1))  # columns x_k - x_0
    det = np.linalg.det(E)
    vol = np.abs(det) / math.factorial(d)
    Einv = np.linalg.inv(E)                 # rows: grad phi_1..phi_d
    grads = np.empty((cells.shape[0], d + 1, d))
    grads[:, 1:, :] = Einv
    grads[:, 0, :] = -Einv.sum(axis=1)
    return vol, grads


def stiffness(coords: np.ndarray, cells: np.ndarray) -> sp.csr_matrix:
    """K_ij = sum_e |e| grad phi_i . grad phi_j, assembled element by element."""
    n = coords.shape[0]
    vol, g = simplex_geometry(coords, cells)
    Ke = vol[:, None, None] * np.einsum("eak,ebk->eab", g, g)
    k = cells.shape[1]
    rows = np.repeat(cells, k, axis=1).ravel()
    cols = np.tile(cells, (1, k)).ravel()
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def lumped_mass(coords, cells, eps) -> np.ndarray:
    """m_i = sum_{e contains i} eps_e |e| / (d+1)."""
    n, k = coords.shape[0], cells.shape[1]
    vol, _ = simplex_geometry(coords, cells)
    eps = np.asarray(eps)
    m = np.zeros(n, dtype=np.result_type(eps.dtype, np.float64))
    for a in range(k):
        np.add.at(m, cells[:, a], eps * vol / k)
    return m


def facet_owner(cells: np.ndarray, bnd: np.ndarray) -> np.ndarray:
    """Index of the cell that owns each boundary facet."""
    m, k = cells.shape
    faces = np.sort(np.concatenate([np.delete(cells, j, axis=1) for j in range(k)]), axis=1)
    fcell = np.tile(np.arange(m, dtype=np.int64), k)
    bs = np.sort(np.asarray(bnd, dtype=faces.dtype), axis=1)
    nf, nb = faces.shape[0], bs.shape[0]
    allk = np.concatenate([faces, bs])
    tag = np.concatenate([np.zeros(nf, np.int8), np.ones(nb, np.int8)])
    # lexicographic order of the vertex triples (pairs in 2D); a boundary
    # facet sorts right after the one cell facet with the same vertices
    order = np.lexsort((tag,) + tuple(allk[:, j] for j in range(k - 2, -1, -1)))
    pos_sorted = np.empty(nf + nb, dtype=np.int64)
    pos_sorted[order] = np.arange(nf + nb)
    pb = pos_sorted[nf:]
    prev = order[pb - 1]
    assert np.all(prev < nf) and np.all(allk[prev] == bs), "boundary facet is not a cell facet"
    return fcell[prev]


def facet_measure(coords: np.ndarray, bnd: np.ndarray) -> np.ndarray:
    """Length (2D) or area (3D) of each boundary facet."""
    x = coords[bnd]
    if coords.shape[1] == 2:
        return np.linalg.norm(x[:, 1] - x[:, 0], axis=1)
    return 0.5 * np.linalg.norm(np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), axis=1)


def abc_damping(coords, cells, bnd, eps, owner=None) -> np.ndarray:
    """D_ii = sum_{F contains i} sqrt(eps_{e(F)}) |F| / d."""
    n, d = coords.shape
    if owner is None:
        owner = facet_owner(cells, bnd)
    eps = np.asarray(eps)
    w = np.sqrt(eps[owner]) * facet_measure(coords, bnd) / d
    D = np.zeros(n, dtype=w.dtype)
    for a in range(d):
        np.add.at(D, bnd[:, a], w)
    return D


def cfl_dt(K: sp.csr_matrix, m: np.ndarray) -> float:
    """2 / sqrt(lam) with lam = max_i sum_j |K_ij| / m_i, a Gershgorin bound on
    the largest eigenvalue of M^-1 K; the leapfrog is stable for dt below it."""
    rowsum = np.asarray(abs(K).sum(axis=1)).ravel()
    lam = np.max(rowsum / np.real(m))
    return 2.0 / math.sqrt(lam)
