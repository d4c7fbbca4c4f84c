"""The first-order flux leapfrog with the split-field layer (App. A) on the
GPU, through the C ABI, against the FP64 oracle: traces with the paper's
square layer (2D) and an anisotropic layer (3D), with and without
conductivity; without layer and conductivity the traces equal the
second-order path with the Neumann boundary; host and device pointers give
the same bits.
"""
import numpy as np
import pytest

from helpers import TRACE_TOL, rel_l2
from oracle import mixed, wave
from workloads import configs, meshes, shots as shots_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg

    return mg


def _dev(x):
    import torch

    return torch.as_tensor(np.asarray(x), dtype=torch.float64, device="cuda:0")


def _square_case():
    m = meshes.square_mesh(8, 2)
    eps = np.random.default_rng(1).uniform(1.0, 3.0, len(m.cells))
    pb = wave.Problem(m.coords, m.cells, m.bnd, eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    f = shots_mod.ricker_frequency(m.mean_edge_length(), 10.0, 1.0)
    nt = 300
    s = shots_mod.ricker(f, dt, nt)
    pts = np.array([[0.0, 0.0], [0.4, -0.2], [-0.5, 0.3]])
    nodes = [int(np.argmin(np.linalg.norm(m.coords - p, axis=1))) for p in pts]
    sh = shots_mod.Shots(np.array(nodes[:2], np.int32), np.array([0, 2, 4], np.int64),
                         np.array([nodes[1], nodes[2], nodes[0], nodes[2]], np.int32))
    return m, eps, dt, s, sh


@pytest.mark.parametrize("with_sigma", [False, True])
def test_square_layer_matches_oracle(mg, with_sigma):
    m, eps, dt, s, sh = _square_case()
    xi, zeta = mixed.square_layer(m.coords, m.cells, 0.7, 1.0, 5.0)
    sigma = 0.5 * eps if with_sigma else None
    ref = mixed.forward(m.coords, m.cells, eps, dt, s, sh.src, sh.rec_ptr, sh.rec,
                        sigma=sigma, xi=xi, zeta=zeta)
    w = configs.Workload("square_pml", m, eps, sh, 1.0, len(s), bc="neumann")
    mesh = mg.mesh_from_workload(w)
    if with_sigma:
        mesh.set_conductivity(sigma)
    y = mg.forward_pml(mesh, _dev(eps), sh, _dev(s), dt, _dev(xi), _dev(zeta)).cpu().numpy()
    assert rel_l2(y, ref) < TRACE_TOL
    yh = mg.forward_pml(mesh, eps, sh, s, dt, xi, zeta)
    assert np.array_equal(y, yh)


def test_no_layer_equals_neumann_leapfrog(mg):
    m, eps, dt, s, sh = _square_case()
    w = configs.Workload("square_pml", m, eps, sh, 1.0, len(s), bc="neumann")
    mesh = mg.mesh_from_workload(w)
    y1 = mg.forward_pml(mesh, _dev(eps), sh, _dev(s), dt).cpu().numpy()
    y2 = mg.forward(mesh, _dev(eps), sh, _dev(s), dt).cpu().numpy()
    assert rel_l2(y1, y2) < TRACE_TOL


def test_3d_anisotropic_layer_matches_oracle(mg):
    w = configs.tiny_3d(nt=80)
    m = w.mesh
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    c = m.coords[m.cells].mean(1)
    zeta = np.where(np.abs(c) > 0.5, 3.0, 0.0)             # per direction
    xi = np.where(np.abs(c).max(1) > 0.5, 3.0, 0.0)
    ref = mixed.forward(m.coords, m.cells, w.eps, dt, s, w.shots.src, w.shots.rec_ptr,
                        w.shots.rec, xi=xi, zeta=zeta)
    mesh = mg.mesh_from_workload(w, bc="neumann")
    y = mg.forward_pml(mesh, _dev(w.eps), w.shots, _dev(s), dt, _dev(xi),
                       _dev(zeta)).cpu().numpy()
    assert rel_l2(y, ref) < TRACE_TOL
