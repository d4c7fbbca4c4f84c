"""Oracle: the paper's first-order leapfrog with element flux variables and
the split-field perfectly matched layer (App. A, Eqs. (system1),
(system2), (leap-frog1), (leap-frog2)), plain FP64 numpy.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module.

Unknowns: p on the nodes (P1) and, per spatial direction k, q^(k) on the
cells (P0).  With A_ii = |T_i|, B^(k)_{ij} = |T_i| d(phi_j)/dx_k on T_i,
C the eps-mass, R the sigma-mass, S the xi-mass (all lumped, as in the rest
of this build) and T^(k) = zeta^(k) A:

    q^(k)_{l+1/2} = q^(k)_{l-1/2} + dt A^-1 (B^(k) p_l - T^(k) q^(k)_{l-1/2})
    p_{l+1}       = p_l + dt C^-1 (f_l - R p_l - S p_l - sum_k B^(k)T q^(k)_{l+1/2})

with p_0 = 0, q_{-1/2} = 0.  The source f is the time integral of the
transmitted wavelet (f_l = dt sum_{m <= l} s_m, so that f_l - f_{l-1} =
dt s_l: the second-order form of wave.py has the source dt^2 s_l).  The
outer boundary is natural (the layer absorbs).  Sample l of a trace is
p_{l+1} at the receiver.  With T = S = R = 0, eliminating q gives exactly
wave.forward with the Neumann boundary.

The layer (Sec. App. A): xi = varsigma where rho1 <= max_k |x_k| <= rho2 and
zeta^(k) = varsigma where rho1 <= |x_k| <= rho2, evaluated here at cell
centroids (reading: the paper gives the functions, not their quadrature).
"""
from __future__ import annotations

import numpy as np

from . import fem


def square_layer(coords, cells, rho1, rho2, varsigma):
    """xi [m] and zeta [m, d] of the paper's layer at the cell centroids."""
    c = np.asarray(coords)[np.asarray(cells)].mean(axis=1)
    a = np.abs(c)
    xi = np.where((a.max(axis=1) >= rho1) & (a.max(axis=1) <= rho2), varsigma, 0.0)
    zeta = np.where((a >= rho1) & (a <= rho2), varsigma, 0.0)
    return xi, zeta


def forward(coords, cells, eps, dt, wavelet, src, rec_ptr, rec, sigma=None, xi=None,
            zeta=None, p0=None, return_states=False):
    """Traces y[r, l] = p_{l+1}[rec[r]] of shot(r) for the first-order scheme;
    p0 ([n, S], optional) replaces the zero initial field (q starts at 0)."""
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    n, d = coords.shape
    m = cells.shape[0]
    vol, grads = fem.simplex_geometry(coords, cells)
    C = fem.lumped_mass(coords, cells, np.asarray(eps, np.float64))
    zeros = np.zeros(m)
    R = fem.lumped_mass(coords, cells, zeros if sigma is None else np.asarray(sigma, float))
    S = fem.lumped_mass(coords, cells, zeros if xi is None else np.asarray(xi, float))
    Z = np.zeros((m, d)) if zeta is None else np.asarray(zeta, float)
    wavelet = np.asarray(wavelet, np.float64)
    nt = len(wavelet)
    src = np.asarray(src, np.int64)
    rec = np.asarray(rec, np.int64)
    rec_ptr = np.asarray(rec_ptr, np.int64)
    S_n = len(src)
    shot = np.repeat(np.arange(S_n), np.diff(rec_ptr))
    p = np.zeros((n, S_n)) if p0 is None else np.array(p0, dtype=np.float64)
    q = np.zeros((d, m, S_n))
    f = np.zeros(S_n)
    y = np.zeros((len(rec), nt))
    states = [p.copy()] if return_states else None
    for l in range(nt):
        f = f + dt * wavelet[l]                     # f_l = dt sum_{m <= l} s_m
        # q^(k) update: (B^(k) p)_e = |e| sum_a dphi_a/dx_k p[cell_a]
        for k in range(d):
            Bp = vol[:, None] * np.einsum("ea,eas->es", grads[:, :, k], p[cells])
            q[k] = q[k] + dt * (Bp - Z[:, k, None] * vol[:, None] * q[k]) / vol[:, None]
        # p update: sum_k B^(k)T q^(k)
        BTq = np.zeros((n, S_n))
        for k in range(d):
            contrib = vol[:, None, None] * grads[:, :, k][:, :, None] * q[k][:, None, :]
            for a in range(d + 1):
                np.add.at(BTq, cells[:, a], contrib[:, a, :])
        rhs = -(R + S)[:, None] * p - BTq
        rhs[src, np.arange(S_n)] += f[np.arange(S_n)]
        p = p + dt * rhs / C[:, None]
        y[:, l] = p[rec, shot]
        if return_states:
            states.append(p.copy())
    return (y, np.array(states)) if return_states else y
