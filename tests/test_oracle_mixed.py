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
