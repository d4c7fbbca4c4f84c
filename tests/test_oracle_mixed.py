"""Pins of the first-order (flux) leapfrog with the split-field layer
(App. A, Eqs. (leap-frog1)-(leap-frog2)).

Facts that do not come from the oracle:
* with T = S = R = 0, eliminating the fluxes gives the second-order scheme:
  the traces equal wave.forward with the Neumann boundary;
* with uniform eps, xi and zeta an eigenvector phi of the lumped pencil
  (K phi = lambda M phi, from a dense generalised eigensolver) evolves as
  p_l = a_l phi, where (a_{l+1}, w_l)
  follows the 2x2 recurrence w_l = (1 - dt zeta) w_{l-1} + dt lambda a_l,
  a_{l+1} = (1 - dt xi/eps) a_l - dt w_l (worked out by hand from the two
  update equations);
* the layer absorbs: the boundary echo at an interior receiver drops below
  a fifth of its value without the layer.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import mixed, wave
from workloads import configs, meshes, shots as shots_mod


def test_without_layer_equals_second_order_scheme():
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=200)
    m, sh = w.mesh, w.shots
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    y2 = wave.forward(pb, dt, s, sh.src, sh.rec_ptr, sh.rec)
    y1 = mixed.forward(m.coords, m.cells, w.eps, dt, s, sh.src, sh.rec_ptr, sh.rec)
    assert np.linalg.norm(y1 - y2) <= 1e-12 * np.linalg.norm(y2)


@pytest.mark.parametrize("mode,xi,zeta", [(1, 0.0, 3.0), (6, 1.5, 0.0), (15, 2.0, 4.0)])
def test_uniform_layer_mode_recurrence(mode, xi, zeta):
    mm = meshes.square_mesh(4, 2)                    # 16x16 squares, 289 nodes
    eps = 2.0
    m_cells = len(mm.cells)
    pb = wave.Problem(mm.coords, mm.cells, mm.bnd, np.full(m_cells, eps), "neumann")
    # an exact eigenpair K phi = lambda M phi of the lumped pencil (dense solver)
    ev, vec = scipy.linalg.eigh(pb.K.toarray(), np.diag(pb.m))
    lam, phi = ev[mode], vec[:, mode]
    assert lam > 0
    dt = 0.5 * pb.cfl_dt()
    nt = 300
    _, P = mixed.forward(mm.coords, mm.cells, np.full(m_cells, eps), dt, np.zeros(nt), [0],
                         [0, 1], [0], xi=np.full(m_cells, xi),
                         zeta=np.full((m_cells, 2), zeta), p0=phi[:, None],
                         return_states=True)
    a, wv = 1.0, 0.0
    scale = np.abs(phi).max()
    for l in range(nt):
        wv = (1 - dt * zeta) * wv + dt * lam * a
        a = (1 - dt * xi / eps) * a - dt * wv
        assert np.abs(P[l + 1, :, 0] - a * phi).max() < 1e-10 * scale * max(1.0, abs(a))


def test_layer_absorbs_boundary_echo():
    mm = meshes.square_mesh(8, 2)
    eps = np.full(len(mm.cells), 1.0)
    pb = wave.Problem(mm.coords, mm.cells, mm.bnd, eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    f = shots_mod.ricker_frequency(mm.mean_edge_length(), 10.0, 1.0)
    t0 = 1.5 / f
    nt = int((t0 + 3.0) / dt)
    s = shots_mod.ricker(f, dt, nt)
    src = int(np.argmin(np.linalg.norm(mm.coords - [0.0, 0.0], axis=1)))
    rec = int(np.argmin(np.linalg.norm(mm.coords - [0.3, 0.0], axis=1)))
    t = (np.arange(nt) + 1) * dt
    ratio = {}
    for vs in (0.0, 5.0):
        xi, zeta = mixed.square_layer(mm.coords, mm.cells, 0.7, 1.0, vs)
        y = mixed.forward(mm.coords, mm.cells, eps, dt, s, [src], [0, 1], [rec], xi=xi,
                          zeta=zeta)[0]
        direct = np.abs(y[(t > t0) & (t < t0 + 0.8)]).max()
        echo = np.abs(y[(t > t0 + 1.3) & (t < t0 + 2.6)]).max()
        ratio[vs] = echo / direct
    assert ratio[5.0] < 0.2 * ratio[0.0]


# ------------------------------------------------------------------ Jacobians
def _layer_case(dim):
    if dim == 2:
        m = meshes.square_mesh(3, 1)
        c = m.coords[m.cells].mean(1)
        xi, zeta = mixed.square_layer(m.coords, m.cells, 0.6, 1.0, 4.0)
    else:
        m = meshes.ellipsoid_mesh(1, (2, 2, 2))
        c = m.coords[m.cells].mean(1)
        zeta = np.where(np.abs(c) > 0.4, 3.0, 0.0)
        xi = np.where(np.abs(c).max(1) > 0.4, 3.0, 0.0)
    rng = np.random.default_rng(dim)
    eps = rng.uniform(1.0, 3.0, len(m.cells))
    sigma = 0.3 * rng.uniform(0.0, 1.0, len(m.cells))
    pb = wave.Problem(m.coords, m.cells, m.bnd, eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    f = shots_mod.ricker_frequency(m.mean_edge_length(), 8.0, 1.0)
    s = shots_mod.ricker(f, dt, 60)
    n = len(m.coords)
    src = rng.choice(n, 2, replace=False)
    rec = rng.choice(n, 5, replace=False)
    return m, eps, sigma, xi, zeta, dt, s, src, np.array([0, 3, 5]), rec


@pytest.mark.parametrize("dim", [2, 3])
def test_pml_tangent_matches_complex_step(dim):
    m, eps, sigma, xi, zeta, dt, s, src, rp, rec = _layer_case(dim)
    de = np.random.default_rng(10 + dim).standard_normal(len(eps))
    h = 1e-30
    yc = mixed.forward(m.coords, m.cells, eps + 1j * h * de, dt, s, src, rp, rec, sigma=sigma,
                       xi=xi, zeta=zeta)
    cs = yc.imag / h
    jv = mixed.tangent(m.coords, m.cells, eps, dt, s, src, rp, rec, de, sigma=sigma, xi=xi,
                       zeta=zeta)
    assert np.abs(cs).max() > 0
    assert np.linalg.norm(jv - cs) <= 1e-12 * np.linalg.norm(cs)


@pytest.mark.parametrize("dim", [2, 3])
def test_pml_adjoint_dot_test(dim):
    m, eps, sigma, xi, zeta, dt, s, src, rp, rec = _layer_case(dim)
    rng = np.random.default_rng(20 + dim)
    de = rng.standard_normal(len(eps))
    W = rng.standard_normal((len(rec), len(s)))
    jv = mixed.tangent(m.coords, m.cells, eps, dt, s, src, rp, rec, de, sigma=sigma, xi=xi,
                       zeta=zeta)
    g = mixed.adjoint_eps(m.coords, m.cells, eps, dt, s, src, rp, rec, W, sigma=sigma, xi=xi,
                          zeta=zeta)
    lhs, rhs = np.sum(jv * W), np.sum(de * g)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.linalg.norm(jv) * np.linalg.norm(W))


def test_pml_jacobians_without_layer_equal_second_order_jacobians():
    """T = S = R = 0: the flux scheme is the second-order scheme with the
    Neumann boundary, so its derivatives are too."""
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=120)
    m, sh = w.mesh, w.shots
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    rng = np.random.default_rng(30)
    de = rng.standard_normal(len(w.eps))
    W = rng.standard_normal((sh.n_traces, len(s)))
    t2 = wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, de)
    t1 = mixed.tangent(m.coords, m.cells, w.eps, dt, s, sh.src, sh.rec_ptr, sh.rec, de)
    assert np.linalg.norm(t1 - t2) <= 1e-10 * np.linalg.norm(t2)
    g2 = wave.adjoint_eps(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, W)
    g1 = mixed.adjoint_eps(m.coords, m.cells, w.eps, dt, s, sh.src, sh.rec_ptr, sh.rec, W)
    assert np.linalg.norm(g1 - g2) <= 1e-10 * np.linalg.norm(g2)
