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

Jacobians with respect to the cell permittivity (only C depends on it):
``tangent`` differentiates every update line by the chain rule
(d(dt rhs / C) = dt drhs / C - dt rhs dC / C^2); ``adjoint_eps`` runs the
reverse-mode recursion of the same lines backwards in time over stored
states and returns g_e = d/deps_e sum_{r,l} w[r,l] y[r,l].

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
    C = fem.lumped_mass(coords, cells, np.asarray(eps))
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
    dtype = np.result_type(np.asarray(eps).dtype, np.float64)   # complex eps: complex step
    p = np.zeros((n, S_n), dtype) if p0 is None else np.array(p0, dtype=dtype)
    q = np.zeros((d, m, S_n), dtype)
    f = np.zeros(S_n)
    y = np.zeros((len(rec), nt), dtype)
    states = [p.copy()] if return_states else None
    for l in range(nt):
        f = f + dt * wavelet[l]                     # f_l = dt sum_{m <= l} s_m
        # q^(k) update: (B^(k) p)_e = |e| sum_a dphi_a/dx_k p[cell_a]
        for k in range(d):
            Bp = vol[:, None] * np.einsum("ea,eas->es", grads[:, :, k], p[cells])
            q[k] = q[k] + dt * (Bp - Z[:, k, None] * vol[:, None] * q[k]) / vol[:, None]
        # p update: sum_k B^(k)T q^(k)
        BTq = np.zeros((n, S_n), dtype)
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


def _operators(coords, cells, eps, sigma, xi, zeta):
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    m = cells.shape[0]
    d = coords.shape[1]
    vol, grads = fem.simplex_geometry(coords, cells)
    C = fem.lumped_mass(coords, cells, np.asarray(eps, np.float64))
    zeros = np.zeros(m)
    R = fem.lumped_mass(coords, cells, zeros if sigma is None else np.asarray(sigma, float))
    S = fem.lumped_mass(coords, cells, zeros if xi is None else np.asarray(xi, float))
    Z = np.zeros((m, d)) if zeta is None else np.asarray(zeta, float)
    return coords, cells, vol, grads, C, R + S, Z


def _grad_p(vol, grads, cells, k, x):
    """(B^(k) x)_e = |e| sum_a dphi_a/dx_k x[cell_a] per cell, per shot."""
    return vol[:, None] * np.einsum("ea,eas->es", grads[:, :, k], x[cells])


def _grad_T(vol, grads, cells, k, y, n):
    """(B^(k)T y)_i = sum_{e contains i} |e| dphi_i/dx_k y_e."""
    out = np.zeros((n, y.shape[1]))
    contrib = vol[:, None, None] * grads[:, :, k][:, :, None] * y[:, None, :]
    for a in range(cells.shape[1]):
        np.add.at(out, cells[:, a], contrib[:, a, :])
    return out


def tangent(coords, cells, eps, dt, wavelet, src, rec_ptr, rec, deps, sigma=None, xi=None,
            zeta=None):
    """Directional derivative of the traces of ``forward`` in the direction
    deps (per finest cell)."""
    coords, cells, vol, grads, C, RS, Z = _operators(coords, cells, eps, sigma, xi, zeta)
    n, d = coords.shape
    m = cells.shape[0]
    dC = fem.lumped_mass(coords, cells, np.asarray(deps, np.float64))
    wavelet = np.asarray(wavelet, np.float64)
    nt = len(wavelet)
    src = np.asarray(src, np.int64)
    rec = np.asarray(rec, np.int64)
    S_n = len(src)
    shot = np.repeat(np.arange(S_n), np.diff(np.asarray(rec_ptr, np.int64)))
    p = np.zeros((n, S_n))
    dp = np.zeros((n, S_n))
    q = np.zeros((d, m, S_n))
    dq = np.zeros((d, m, S_n))
    f = np.zeros(S_n)
    y = np.zeros((len(rec), nt))
    for l in range(nt):
        f = f + dt * wavelet[l]
        for k in range(d):
            q[k] = q[k] + dt * (_grad_p(vol, grads, cells, k, p) -
                                Z[:, k, None] * vol[:, None] * q[k]) / vol[:, None]
            dq[k] = dq[k] + dt * (_grad_p(vol, grads, cells, k, dp) -
                                  Z[:, k, None] * vol[:, None] * dq[k]) / vol[:, None]
        rhs = -RS[:, None] * p - sum(_grad_T(vol, grads, cells, k, q[k], n) for k in range(d))
        rhs[src, np.arange(S_n)] += f
        drhs = -RS[:, None] * dp - sum(_grad_T(vol, grads, cells, k, dq[k], n)
                                       for k in range(d))
        dp = dp + dt * drhs / C[:, None] - dt * rhs * (dC / C ** 2)[:, None]
        p = p + dt * rhs / C[:, None]
        y[:, l] = dp[rec, shot]
    return y


def adjoint_eps(coords, cells, eps, dt, wavelet, src, rec_ptr, rec, W, sigma=None, xi=None,
                zeta=None):
    """g_e = d/deps_e sum_{r,l} W[r,l] y[r,l] for the traces of ``forward``.

    Step l maps (p_l, q_{l-1/2}) to q_{l+1/2} = (1 - dt zeta) q + dt B p_l / |e|,
    then p_{l+1} = p_l + dt rhs_l / C with rhs_l = f_l e - (R+S) p_l -
    sum_k B^(k)T q^(k)_{l+1/2}.  Going back from l = nt-1, with a the adjoint
    of p_{l+1} (its objective term w_l at the receivers plus what step l+1
    sends back) and b that of q_{l+1/2} sent back by step l+1: the
    C-sensitivity gains -dt rhs_l a / C^2; the adjoint of rhs_l is
    r = a dt / C; the full adjoint of q^(k)_{l+1/2} is Q_k = b_k - B^(k) r;
    p_l receives a - (R+S) r + dt sum_k B^(k)T (Q_k / |e|) and q_{l-1/2}
    receives (1 - dt zeta_k) Q_k.  C_i = sum_{e contains i} eps_e |e| / (d+1)
    turns the C-sensitivity into the cell gradient."""
    coords, cells, vol, grads, C, RS, Z = _operators(coords, cells, eps, sigma, xi, zeta)
    n, d = coords.shape
    m = cells.shape[0]
    wavelet = np.asarray(wavelet, np.float64)
    nt = len(wavelet)
    src = np.asarray(src, np.int64)
    rec = np.asarray(rec, np.int64)
    S_n = len(src)
    shot = np.repeat(np.arange(S_n), np.diff(np.asarray(rec_ptr, np.int64)))
    W = np.asarray(W, np.float64)
    # forward, keeping p_l and rhs_l
    p = np.zeros((n, S_n))
    q = np.zeros((d, m, S_n))
    f = np.zeros(S_n)
    P, RHS = [], []
    for l in range(nt):
        f = f + dt * wavelet[l]
        for k in range(d):
            q[k] = q[k] + dt * (_grad_p(vol, grads, cells, k, p) -
                                Z[:, k, None] * vol[:, None] * q[k]) / vol[:, None]
        rhs = -RS[:, None] * p - sum(_grad_T(vol, grads, cells, k, q[k], n) for k in range(d))
        rhs[src, np.arange(S_n)] += f
        P.append(p.copy())
        RHS.append(rhs)
        p = p + dt * rhs / C[:, None]
    a = np.zeros((n, S_n))          # adjoint of p_{l+1} sent back by step l+1
    b = np.zeros((d, m, S_n))       # adjoint of q_{l+1/2} sent back by step l+1
    gC = np.zeros(n)
    for l in range(nt - 1, -1, -1):
        A = a.copy()
        np.add.at(A, (rec, shot), W[:, l])
        gC += np.sum(-dt * RHS[l] * A, axis=1) / C ** 2
        Ar = A * dt / C[:, None]
        to_p = A - RS[:, None] * Ar
        for k in range(d):
            Qk = b[k] - _grad_p(vol, grads, cells, k, Ar)
            to_p = to_p + dt * _grad_T(vol, grads, cells, k, Qk / vol[:, None], n)
            b[k] = (1.0 - dt * Z[:, k, None]) * Qk
        a = to_p
    k1 = cells.shape[1]
    return (vol / k1) * gC[cells].sum(axis=1)
