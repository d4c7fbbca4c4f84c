"""Oracle: explicit leapfrog wave propagation, its tangent and its adjoint,
in plain FP64 numpy/scipy.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module.

The scheme (App. A, Eqs. (leap-frog1)-(leap-frog2)) with the flux q
eliminated (so sum_k B^T A^-1 B = K), the mass lumped, the split-field PML
replaced by the first-order absorbing boundary D, and the source driven by
the wavelet samples s_l:

    (M + dt/2 D) p_{l+1} = 2 M p_l - (M - dt/2 D) p_{l-1} - dt^2 (K p_l - s_l e_src)

for l = 0..nt-1 with p_0 = p_{-1} = 0.  Sample l of the trace of a receiver
node r is p_{l+1}[r].  Each shot is an independent column of the state.

Tangent: the derivative of the scheme w.r.t. eps in a direction deps; this
is the auxiliary system of Eqs. (aku_ankka), (linearized1)-(linearized2)
with the source built from the lumped dM/deps and dD/deps.

Adjoint: the transpose of the tangent map, obtained from the Lagrangian of
the residual form above; it gives grad_eps <w, y(eps)> for trace weights w.
The per-fine-cell gradient is restricted to a coarse level through the
nesting map, because the permittivity is a sum of coarse-cell indicators
(Sec. II-B, eps_r = sum_j c_j chi'_j).

Boundary modes: "abc" (D as above), "neumann" (D = 0) and "dirichlet"
(D = 0 and boundary nodes held at zero after every step).

Conductivity (optional): the sigma du/dt term of Eq. (pde1), i.e. the mass
matrix R of App. A weighted by sigma, lumped like the eps-mass
(R_ii = sum_{e contains i} sigma_e |e|/(d+1)), joins the damping and is
centred in time with it: D above becomes D + R.  sigma is a fixed nuisance
parameter (Sec. III): the tangent and the adjoint differentiate with respect
to eps only.
"""
from __future__ import annotations

import numpy as np

from . import fem


class Problem:
    """Assembled FP64 system for one mesh, permittivity and boundary mode."""

    def __init__(self, coords, cells, bnd, eps, bc="abc", sigma=None):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.bnd = np.asarray(bnd, dtype=np.int64)
        self.eps = np.asarray(eps)
        self.bc = bc
        self.n, self.d = self.coords.shape
        self.K = fem.stiffness(self.coords, self.cells)
        self.vol, _ = fem.simplex_geometry(self.coords, self.cells)
        self.m = fem.lumped_mass(self.coords, self.cells, self.eps)
        self.owner = fem.facet_owner(self.cells, self.bnd)
        self.fmeas = fem.facet_measure(self.coords, self.bnd)
        if bc == "abc":
            self.D = fem.abc_damping(self.coords, self.cells, self.bnd, self.eps,
                                     self.owner)
        elif bc in ("neumann", "dirichlet"):
            self.D = np.zeros(self.n, dtype=self.m.dtype)
        else:
            raise ValueError(bc)
        # lumped conductivity mass R, added to the damping
        self.R = (np.zeros(self.n) if sigma is None
                  else fem.lumped_mass(self.coords, self.cells, np.asarray(sigma, np.float64)))
        self.D = self.D + self.R
        self.fixed = (np.unique(self.bnd.ravel()) if bc == "dirichlet"
                      else np.zeros(0, dtype=np.int64))

    def cfl_dt(self) -> float:
        return fem.cfl_dt(self.K, self.m)

    # -- derivative pieces -------------------------------------------------
    def dmass(self, deps):
        """dm_i = sum_{e contains i} deps_e |e|/(d+1)."""
        k = self.d + 1
        out = np.zeros(self.n, dtype=np.result_type(deps, np.float64))
        for a in range(k):
            np.add.at(out, self.cells[:, a], deps * self.vol / k)
        return out

    def ddamp(self, deps):
        """dD_ii = sum_{F contains i} deps_{e(F)} |F| / (2 d sqrt(eps_{e(F)}))."""
        out = np.zeros(self.n, dtype=np.result_type(deps, self.eps, np.float64))
        if self.bc != "abc":
            return out
        e = self.owner
        w = deps[e] * self.fmeas / (2.0 * self.d * np.sqrt(self.eps[e]))
        for a in range(self.d):
            np.add.at(out, self.bnd[:, a], w)
        return out


def _shot_of_trace(rec_ptr):
    rec_ptr = np.asarray(rec_ptr, dtype=np.int64)
    return np.repeat(np.arange(len(rec_ptr) - 1), np.diff(rec_ptr))


def forward(pb: Problem, dt, wavelet, src, rec_ptr, rec, nt=None, p0=None,
            pm1=None, return_states=False):
    """Traces y[r, l] = p_{l+1}[rec[r], shot(r)], l = 0..nt-1.

    p0, pm1 (optional [n, S]) replace the zero initial states.
    If return_states, also returns the states p_{-1}..p_nt as [nt+2, n, S]."""
    wavelet = np.asarray(wavelet)
    nt = len(wavelet) if nt is None else nt
    src = np.asarray(src, dtype=np.int64)
    rec = np.asarray(rec, dtype=np.int64)
    S = len(src)
    shot = _shot_of_trace(rec_ptr)
    dtype = np.result_type(pb.m.dtype, wavelet.dtype, np.float64)
    A = (pb.m + 0.5 * dt * pb.D)[:, None]
    B = (pb.m - 0.5 * dt * pb.D)[:, None]
    M2 = (2.0 * pb.m)[:, None]
    p = np.zeros((pb.n, S), dtype) if p0 is None else np.array(p0, dtype=dtype)
    pm = np.zeros((pb.n, S), dtype) if pm1 is None else np.array(pm1, dtype=dtype)
    y = np.zeros((len(rec), nt), dtype)
    states = None
    if return_states:
        states = np.zeros((nt + 2, pb.n, S), dtype)
        states[0], states[1] = pm, p
    cols = np.arange(S)
    for l in range(nt):
        rhs = M2 * p - B * pm - dt * dt * (pb.K @ p)
        rhs[src, cols] += dt * dt * wavelet[l]
        pn = rhs / A
        pn[pb.fixed, :] = 0.0
        y[:, l] = pn[rec, shot]
        pm, p = p, pn
        if return_states:
            states[l + 2] = p
    return (y, states) if return_states else y


def tangent(pb: Problem, dt, wavelet, src, rec_ptr, rec, deps, nt=None):
    """Directional derivative dy = (dy/deps) deps of the traces."""
    wavelet = np.asarray(wavelet)
    nt = len(wavelet) if nt is None else nt
    src = np.asarray(src, dtype=np.int64)
    rec = np.asarray(rec, dtype=np.int64)
    S = len(src)
    shot = _shot_of_trace(rec_ptr)
    dm = pb.dmass(deps)[:, None]
    dD = pb.ddamp(deps)[:, None]
    A = (pb.m + 0.5 * dt * pb.D)[:, None]
    B = (pb.m - 0.5 * dt * pb.D)[:, None]
    M2 = (2.0 * pb.m)[:, None]
    dtype = np.result_type(pb.m.dtype, dm.dtype, np.float64)
    p = np.zeros((pb.n, S), dtype)
    pm = np.zeros((pb.n, S), dtype)
    q = np.zeros((pb.n, S), dtype)
    qm = np.zeros((pb.n, S), dtype)
    dy = np.zeros((len(rec), nt), dtype)
    cols = np.arange(S)
    for l in range(nt):
        rhs = M2 * p - B * pm - dt * dt * (pb.K @ p)
        rhs[src, cols] += dt * dt * wavelet[l]
        pn = rhs / A
        pn[pb.fixed, :] = 0.0
        # derivative of the residual (M + dt/2 D) p+ - 2M p + (M - dt/2 D) p-
        src_t = dm * (pn - 2.0 * p + pm) + 0.5 * dt * dD * (pn - pm)
        qn = (M2 * q - B * qm - dt * dt * (pb.K @ q) - src_t) / A
        qn[pb.fixed, :] = 0.0
        dy[:, l] = qn[rec, shot]
        pm, p = p, pn
        qm, q = q, qn
    return dy


def adjoint_eps(pb: Problem, dt, wavelet, src, rec_ptr, rec, w, nt=None):
    """Gradient g_e = d/deps_e sum_{r,l} w[r,l] y[r,l] per finest cell.

    Multipliers mu_l (l = 0..nt-1) of the residual rows
      F_l = (M + dt/2 D) p_{l+1} - (2M - dt^2 K) p_l + (M - dt/2 D) p_{l-1} - dt^2 s_l e
    satisfy, for k = nt..1 with mu_nt = mu_{nt+1} = 0,
      (M + dt/2 D) mu_{k-1} = (2M - dt^2 K) mu_k - (M - dt/2 D) mu_{k+1} + R^T w_{k-1},
    and g_e = -sum_l mu_l^T dF_l/deps_e with
      dF_l/deps_e = dM/deps_e (p_{l+1} - 2 p_l + p_{l-1}) + dt/2 dD/deps_e (p_{l+1} - p_{l-1}).
    """
    wavelet = np.asarray(wavelet)
    nt = len(wavelet) if nt is None else nt
    src = np.asarray(src, dtype=np.int64)
    rec = np.asarray(rec, dtype=np.int64)
    S = len(src)
    shot = _shot_of_trace(rec_ptr)
    _, P = forward(pb, dt, wavelet, src, rec_ptr, rec, nt, return_states=True)
    # P[l + 1] = p_l for l = -1..nt
    A = (pb.m + 0.5 * dt * pb.D)[:, None]
    B = (pb.m - 0.5 * dt * pb.D)[:, None]
    M2 = (2.0 * pb.m)[:, None]
    mu_k = np.zeros((pb.n, S))
    mu_k1 = np.zeros((pb.n, S))
    # node-wise accumulations of mu_l (second difference) and mu_l (centred difference)
    Gn = np.zeros(pb.n)
    Hn = np.zeros(pb.n)
    for k in range(nt, 0, -1):
        rhs = M2 * mu_k - B * mu_k1 - dt * dt * (pb.K @ mu_k)
        np.add.at(rhs, (rec, shot), w[:, k - 1])
        mu = rhs / A
        mu[pb.fixed, :] = 0.0
        l = k - 1
        p_next, p_cur, p_prev = P[l + 2], P[l + 1], P[l]
        Gn += (mu * (p_next - 2.0 * p_cur + p_prev)).sum(axis=1)
        Hn += (mu * (p_next - p_prev)).sum(axis=1)
        mu_k1, mu_k = mu_k, mu
    return cell_gradient(pb, dt, Gn, Hn)


def cell_gradient(pb: Problem, dt, Gn, Hn):
    """g_e = -(|e|/(d+1)) sum_{i in e} G_i
             - (dt/2) sum_{F in e, F on boundary} |F|/(2 d sqrt(eps_e)) sum_{i in F} H_i."""
    k = pb.d + 1
    g = -(pb.vol / k) * Gn[pb.cells].sum(axis=1)
    if pb.bc == "abc":
        e = pb.owner
        wF = pb.fmeas / (2.0 * pb.d * np.sqrt(np.real(pb.eps[e])))
        np.add.at(g, e, -0.5 * dt * wF * Hn[pb.bnd].sum(axis=1))
    return g


def restrict(g_fine, ancestor, n_coarse):
    """g_c = sum over fine cells e whose ancestor is c of g_e."""
    out = np.zeros(n_coarse)
    np.add.at(out, np.asarray(ancestor, dtype=np.int64), g_fine)
    return out


def prolong(v_coarse, ancestor):
    """deps_e = v_{anc(e)} (the nested piecewise-constant parameterisation)."""
    return np.asarray(v_coarse)[np.asarray(ancestor, dtype=np.int64)]
