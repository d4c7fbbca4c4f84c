"""Pins of the oracle's conductivity term (the sigma du/dt of Eq. (pde1),
lumped sigma-mass R centred in time with the boundary damping).

Facts that do not come from the oracle:
* a Dirichlet eigenmode of the uniform grid with homogeneous eps and sigma
  evolves exactly as r^l cos(l theta) phi, the solution of the damped
  three-term recurrence: r^2 = (1 - c)/(1 + c), c = dt sigma / (2 eps),
  cos theta = (2 - dt^2 lambda) / (2 sqrt(1 - c^2));
* with sigma = kappa eps the lumped sigma-mass is kappa times the (pinned)
  eps-mass, and the discrete energy changes by exactly
  -(p_{l+1} - p_{l-1})^T kappa M (p_{l+1} - p_{l-1}) / (4 dt) per step;
* the eps-tangent and eps-adjoint stay exact derivatives with sigma on
  (complex step, dot test).
"""
import math

import numpy as np
import pytest

from oracle import wave
from workloads import configs, meshes


def _energy(pb, dt, p1, p0):
    v = (p1 - p0) / dt
    return 0.5 * float(np.sum(v * (pb.m[:, None] * v))) + 0.5 * float(np.sum(p1 * (pb.K @ p0)))


@pytest.mark.parametrize("mode", [(1, 1), (3, 2)])
def test_damped_dirichlet_eigenmode_closed_form(mode):
    a, b = mode
    m = meshes.square_mesh(8, 3)                    # 64x64 squares, h = 1/32
    h, eps, sig = 2.0 / 64, 3.0, 0.8
    pb = wave.Problem(m.coords, m.cells, m.bnd, np.full(len(m.cells), eps), "dirichlet",
                      sigma=np.full(len(m.cells), sig))
    dt = 0.5 * pb.cfl_dt()
    x, y = m.coords[:, 0], m.coords[:, 1]
    phi = np.sin(a * math.pi * (x + 1) / 2) * np.sin(b * math.pi * (y + 1) / 2)
    lam = (4.0 / h ** 2) * (math.sin(a * math.pi * h / 4) ** 2
                           + math.sin(b * math.pi * h / 4) ** 2) / eps
    c = 0.5 * dt * sig / eps
    r = math.sqrt((1 - c) / (1 + c))
    th = math.acos((2 - dt * dt * lam) / (2 * math.sqrt(1 - c * c)))
    nt = 600
    _, P = wave.forward(pb, dt, np.zeros(nt), [0], [0, 1], [0], p0=phi[:, None],
                        pm1=(math.cos(th) / r * phi)[:, None], return_states=True)
    for l in range(-1, nt + 1):
        assert np.abs(P[l + 1, :, 0] - r ** l * math.cos(l * th) * phi).max() < 1e-11
    assert r ** nt < 0.9                              # the damping is visible


def test_energy_loss_of_conductivity():
    w = configs.tiny_2d(n_coarse=4, n_refine=2)
    kappa = 2.0
    pb = wave.Problem(w.mesh.coords, w.mesh.cells, w.mesh.bnd, w.eps, "neumann",
                      sigma=kappa * w.eps)
    dt = 0.5 * pb.cfl_dt()
    x, y = w.mesh.coords[:, 0], w.mesh.coords[:, 1]
    p0 = np.exp(-((x - 0.2) ** 2 + (y + 0.1) ** 2) / 0.05)[:, None]
    nt = 400
    _, P = wave.forward(pb, dt, np.zeros(nt), [0], [0, 1], [0], p0=p0, pm1=p0,
                        return_states=True)
    E0 = _energy(pb, dt, P[1], P[0])
    for l in range(1, nt + 1):
        dE = _energy(pb, dt, P[l + 1], P[l]) - _energy(pb, dt, P[l], P[l - 1])
        jump = P[l + 1] - P[l - 1]
        loss = -np.sum(jump * (kappa * pb.m[:, None] * jump)) / (4.0 * dt)
        assert abs(dE - loss) < 1e-12 * E0
    assert _energy(pb, dt, P[-1], P[-2]) < 0.5 * E0


def test_eps_derivatives_with_conductivity():
    w = configs.tiny_2d()
    sig = np.random.default_rng(9).uniform(0.0, 3.0, len(w.eps))
    m, sh = w.mesh, w.shots
    mk = lambda eps: wave.Problem(m.coords, m.cells, m.bnd, eps, w.bc, sigma=sig)
    pb = mk(w.eps)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    rng = np.random.default_rng(10)
    de = rng.standard_normal(len(w.eps))
    dy = wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, de)
    h = 1e-20
    cs = wave.forward(mk(w.eps + 1j * h * de), dt, s, sh.src, sh.rec_ptr, sh.rec).imag / h
    assert np.linalg.norm(dy - cs) <= 1e-12 * np.linalg.norm(cs)
    W = rng.standard_normal((sh.n_traces, len(s)))
    g = wave.adjoint_eps(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, W)
    lhs, rhs = np.sum(dy * W), np.sum(de * g)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.linalg.norm(dy) * np.linalg.norm(W))
    # sigma changes the traces (the term is not dropped)
    y0 = wave.forward(wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc), dt, s, sh.src,
                      sh.rec_ptr, sh.rec)
    y1 = wave.forward(pb, dt, s, sh.src, sh.rec_ptr, sh.rec)
    assert np.linalg.norm(y1 - y0) > 1e-3 * np.linalg.norm(y0)
