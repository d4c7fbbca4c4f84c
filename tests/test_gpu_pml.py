"""The first-order flux leapfrog with the split-field layer (App. A) on the
GPU, through the C ABI, against the FP64 oracle: traces with the paper's
square layer (2D) and an anisotropic layer (3D), with and without
conductivity; without layer and conductivity the traces equal the
second-order path with the Neumann boundary; host and device pointers give
the same bits.  Its Jacobians: J v and J^T w on a level against the
oracle's tangent and adjoint (Jacobian tolerance), the dot test on the GPU
outputs, checkpoint spacing that leaves J^T w's bits unchanged, and equality
with the second-order Jacobians without layer.
"""
import numpy as np
import pytest

from helpers import JAC_TOL, TRACE_TOL, rel_l2
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


def _jac_refs(m, eps, dt, s, sh, level, v, W, sigma=None, xi=None, zeta=None):
    anc = m.ancestor(level)
    jv = mixed.tangent(m.coords, m.cells, eps, dt, s, sh.src, sh.rec_ptr, sh.rec,
                       wave.prolong(v, anc), sigma=sigma, xi=xi, zeta=zeta)
    g = mixed.adjoint_eps(m.coords, m.cells, eps, dt, s, sh.src, sh.rec_ptr, sh.rec, W,
                          sigma=sigma, xi=xi, zeta=zeta)
    return jv, wave.restrict(g, anc, m.n_cells[level])


@pytest.mark.parametrize("with_sigma", [False, True])
def test_square_layer_jacobians_match_oracle(mg, with_sigma):
    import torch

    m, eps, dt, s, sh = _square_case()
    xi, zeta = mixed.square_layer(m.coords, m.cells, 0.7, 1.0, 5.0)
    sigma = 0.5 * eps if with_sigma else None
    rng = np.random.default_rng(7)
    level = 1
    v = rng.standard_normal(m.n_cells[level])
    W = rng.standard_normal((sh.n_traces, len(s))).astype(np.float32)
    ref_jv, ref_g = _jac_refs(m, eps, dt, s, sh, level, v, W.astype(np.float64), sigma, xi, zeta)
    w = configs.Workload("square_pml", m, eps, sh, 1.0, len(s), bc="neumann")
    mesh = mg.mesh_from_workload(w)
    if with_sigma:
        mesh.set_conductivity(sigma)
    jv = mg.jacobian_apply_pml(mesh, level, _dev(eps), sh, _dev(s), dt, _dev(v), _dev(xi),
                               _dev(zeta)).cpu().numpy()
    assert rel_l2(jv, ref_jv) < JAC_TOL
    Wd = torch.as_tensor(W, device="cuda:0")
    g = mg.jacobian_T_apply_pml(mesh, level, _dev(eps), sh, _dev(s), dt, Wd, _dev(xi), _dev(zeta),
                                ckpt_every=32).cpu().numpy()
    assert rel_l2(g, ref_g) < JAC_TOL
    # dot test on the GPU outputs, inner products in FP64
    lhs = float(np.sum(jv.astype(np.float64) * W))
    rhs = float(np.sum(v * g))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    # checkpoint spacing changes nothing; host pointers give the same bits
    g7 = mg.jacobian_T_apply_pml(mesh, level, _dev(eps), sh, _dev(s), dt, Wd, _dev(xi),
                                 _dev(zeta), ckpt_every=7).cpu().numpy()
    assert np.array_equal(g7, g)
    # one segment: the forward keeps every state and nothing is recomputed
    gk = mg.jacobian_T_apply_pml(mesh, level, _dev(eps), sh, _dev(s), dt, Wd, _dev(xi),
                                 _dev(zeta), ckpt_every=len(s)).cpu().numpy()
    assert np.array_equal(gk, g)
    gh = mg.jacobian_T_apply_pml(mesh, level, eps, sh, s, dt, W, xi, zeta, ckpt_every=32)
    assert np.array_equal(gh, g)
    jh = mg.jacobian_apply_pml(mesh, level, eps, sh, s, dt, v, xi, zeta)
    assert np.array_equal(jh, jv)


def test_3d_layer_jacobians_match_oracle(mg):
    import torch

    w = configs.tiny_3d(nt=80)
    m = w.mesh
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    c = m.coords[m.cells].mean(1)
    zeta = np.where(np.abs(c) > 0.5, 3.0, 0.0)
    xi = np.where(np.abs(c).max(1) > 0.5, 3.0, 0.0)
    rng = np.random.default_rng(8)
    level = 0
    v = rng.standard_normal(m.n_cells[level])
    W = rng.standard_normal((w.shots.n_traces, len(s))).astype(np.float32)
    ref_jv, ref_g = _jac_refs(m, w.eps, dt, s, w.shots, level, v, W.astype(np.float64), None,
                              xi, zeta)
    mesh = mg.mesh_from_workload(w, bc="neumann")
    jv = mg.jacobian_apply_pml(mesh, level, _dev(w.eps), w.shots, _dev(s), dt, _dev(v),
                               _dev(xi), _dev(zeta)).cpu().numpy()
    assert rel_l2(jv, ref_jv) < JAC_TOL
    g = mg.jacobian_T_apply_pml(mesh, level, _dev(w.eps), w.shots, _dev(s), dt,
                                torch.as_tensor(W, device="cuda:0"), _dev(xi), _dev(zeta),
                                ckpt_every=16).cpu().numpy()
    assert rel_l2(g, ref_g) < JAC_TOL


def test_jacobians_without_layer_equal_second_order_jacobians(mg):
    import torch

    m, eps, dt, s, sh = _square_case()
    w = configs.Workload("square_pml", m, eps, sh, 1.0, len(s), bc="neumann")
    mesh = mg.mesh_from_workload(w)
    rng = np.random.default_rng(9)
    v = rng.standard_normal(m.n_cells[1])
    W = torch.as_tensor(rng.standard_normal((sh.n_traces, len(s))).astype(np.float32),
                        device="cuda:0")
    j1 = mg.jacobian_apply_pml(mesh, 1, _dev(eps), sh, _dev(s), dt, _dev(v)).cpu().numpy()
    j2 = mg.jacobian_apply(mesh, 1, _dev(eps), sh, _dev(s), dt, _dev(v)).cpu().numpy()
    assert rel_l2(j1, j2) < JAC_TOL
    g1 = mg.jacobian_T_apply_pml(mesh, 1, _dev(eps), sh, _dev(s), dt, W).cpu().numpy()
    g2 = mg.jacobian_T_apply(mesh, 1, _dev(eps), sh, _dev(s), dt, W).cpu().numpy()
    assert rel_l2(g1, g2) < JAC_TOL


def test_graph_chunks_give_the_same_bits(mg):
    """The PML drivers replay whole chunks of steps as CUDA graphs (the step
    index and the state slots read from a device base the graph moves):
    forward, J v and J^T w (checkpoint spacings with a shorter last
    segment, and the single kept segment) carry the bits of plain launches
    (MG_NO_GRAPH), with chunks that leave remainders."""
    import torch
    from paper_1707_04605_gb300 import _lib as L

    m, eps, dt, s, sh = _square_case()
    xi, zeta = mixed.square_layer(m.coords, m.cells, 0.7, 1.0, 5.0)
    w = configs.Workload("square_pml", m, eps, sh, 1.0, len(s), bc="neumann")
    mesh = mg.mesh_from_workload(w)
    rng = np.random.default_rng(21)
    v = _dev(rng.standard_normal(m.n_cells[1]))
    W = torch.as_tensor(rng.standard_normal((sh.n_traces, len(s))).astype(np.float32),
                        device="cuda:0")
    args = (_dev(eps), sh, _dev(s), dt)
    lay = (_dev(xi), _dev(zeta))

    def run(flags, ck):
        return (mg.forward_pml(mesh, *args, *lay, flags=flags),
                mg.jacobian_apply_pml(mesh, 1, *args, v, *lay, flags=flags),
                mg.jacobian_T_apply_pml(mesh, 1, *args, W, *lay, ckpt_every=ck, flags=flags))

    for chunk in (128, 16):
        mesh.set_tuning(chunk=chunk)
        for ck in (32, 7, len(s)):
            ref = run(L.MG_NO_GRAPH, ck)
            out = run(0, ck)
            for a, b in zip(ref, out):
                assert torch.equal(a, b), (chunk, ck)
