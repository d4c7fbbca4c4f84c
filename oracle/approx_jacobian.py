"""Oracle: the paper's approximate Jacobian (App. A.1-A.3: auxiliary
system, Green's function and reciprocity, multigrid approach), FP64 numpy.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module.

The leapfrog of wave.py is a linear time-invariant system: with
A(z) = (M + dt/2 D) z - 2M + (M - dt/2 D) z^-1 + dt^2 K, a source sequence
s_l at node i gives p_{l+1}[r] = sum_k H_{r,i}[l - k] s_k with
H(z) = dt^2 A(z)^-1.  A(z) is symmetric, so H_{r,i} = H_{i,r}
(reciprocity).  The tangent recursion is the same system driven, at every
node i, by the auxiliary source (Eqs. (aku_ankka), (linearized1)-(linearized2),
written for the second-order form)

    s^(i)_l = -[dm_i (p_{l+1} - 2 p_l + p_{l-1})_i + (dt/2) dd_i (p_{l+1} - p_{l-1})_i] / dt^2,

so the trace derivative at receiver r is sum_i H_{r,i} * s^(i) (approx_1,
Eq. (approx_1): exact by linearity).  Steps (1)-(4) of App. A.2 obtain the
Green's functions H_{i,r} = H_{r,i} from a forward run with the source at r
recorded at node i; here that run is driven by a unit impulse (s_0 = 1),
which gives H exactly (reading: the paper deconvolves a wavelet run with
Tikhonov regularisation; on truncated traces and a Ricker wavelet whose
leading samples are ~1e-8 of its peak that estimate was off by order one
in this discretisation, while the impulse run costs one forward and is
exact).

approx_2 (multigrid, Eq. (approx_2)): the auxiliary sources of coarse cell
j sit on its d+1 corner nodes only, with the lumped coarse mass
dm'_i = |T'_j| / (d+1) (reading: the paper's consistent coarse mass C' is
lumped, as the fine mass is here) and no boundary-damping term (the paper's
auxiliary source carries dC/dc only).  Per unit coarse mass the response of
node i is phi_i = H_{r,i} * (-(p_{l+1} - 2 p_l + p_{l-1})_i / dt^2), and the
column of cell j is (|T'_j| / (d+1)) sum_{i in corners(j)} phi_i.
"""
from __future__ import annotations

import numpy as np

from . import wave


def states(pb, dt, wavelet, node):
    """p_l at every node for l = -1..nt, the source sequence at `node`: [nt+2, n]."""
    _, P = wave.forward(pb, dt, wavelet, [node], [0, 1], [node], return_states=True)
    return P[:, :, 0]


def greens(pb, dt, nt: int, r):
    """Impulse responses H_{i,r}[k] = p_{k+1}[i] of a unit impulse at r
    (s_0 = 1), k = 0..nt-1, for every node i: [n, nt]."""
    imp = np.zeros(nt)
    imp[0] = 1.0
    return states(pb, dt, imp, r)[2:].T


def aux_sources(P, dt, dm, dd):
    """s^(i)_l for every node (rows) from the states P [nt+2, n]."""
    d2 = P[2:] - 2.0 * P[1:-1] + P[:-2]           # p_{l+1} - 2 p_l + p_{l-1}
    d1 = P[2:] - P[:-2]
    return (-(dm[None, :] * d2 + 0.5 * dt * dd[None, :] * d1) / dt ** 2).T


def convolve_causal(g, s):
    """Per row, sum_k g[l-k] s[k] for l = 0..nt-1: [rows, nt]."""
    nt = g.shape[1]
    out = np.zeros((g.shape[0], nt))
    for i in range(g.shape[0]):
        out[i] = np.convolve(g[i], s[i])[:nt]
    return out


def approx1_column(pb, dt, wavelet, src, rec, deps):
    """approx_1: trace derivative at `rec` (source at `src`) in the direction
    deps of the finest-cell permittivity; every node contributes."""
    P = states(pb, dt, wavelet, src)
    g = greens(pb, dt, len(wavelet), rec)
    s = aux_sources(P, dt, pb.dmass(deps), pb.ddamp(deps))
    return convolve_causal(g, s).sum(0)


def coarse_corners(cells, ancestor, n_level):
    """Corner nodes of every level cell: the descendant vertices used by
    exactly one descendant (regular refinement keeps each corner in a single
    child).  [n_level, d+1] int."""
    k = cells.shape[1]
    out = np.zeros((n_level, k), dtype=np.int64)
    for c in range(n_level):
        v, cnt = np.unique(cells[ancestor == c].ravel(), return_counts=True)
        corners = v[cnt == 1]
        if len(corners) != k:
            raise ValueError("level cell without d+1 single-use corners")
        out[c] = corners
    return out


def node_responses(pb, dt, wavelet, src, rec, nodes):
    """phi_i = H_{rec,i} * (-(p_{l+1} - 2 p_l + p_{l-1})_i / dt^2) for the
    given nodes: [len(nodes), nt]."""
    P = states(pb, dt, wavelet, src)
    g = greens(pb, dt, len(wavelet), rec)
    unit = np.ones(pb.n)
    s = aux_sources(P, dt, unit, np.zeros(pb.n))
    return convolve_causal(g[nodes], s[nodes])


def approx2_columns(pb, dt, wavelet, src, rec, corners, vol_level):
    """approx_2 trace derivatives at `rec` for every level cell: [n_level, nt]."""
    nodes = np.unique(corners)
    phi = node_responses(pb, dt, wavelet, src, rec, nodes)
    row = {int(v): i for i, v in enumerate(nodes)}
    k = corners.shape[1]
    out = np.zeros((corners.shape[0], len(wavelet)))
    for c in range(corners.shape[0]):
        for v in corners[c]:
            out[c] += vol_level[c] / k * phi[row[int(v)]]
    return out
