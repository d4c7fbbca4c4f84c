"""The paper's approximate Jacobian (App. A.1-A.3) on the GPU, through the C
ABI: node responses and projected columns against the FP64 oracle (same
algorithm: impulse Green's functions, corner auxiliary sources, lumped
coarse mass), and, at the finest level with a Neumann boundary (where the
approximation is exact), against the GPU's exact tangent.
"""
import numpy as np
import pytest

from helpers import rel_l2
from oracle import approx_jacobian as aj
from oracle import projected as oproj
from oracle import wave
from workloads import configs, shots as shots_mod

pytestmark = pytest.mark.gpu

TOL = 1e-4   # FP32 forward runs and FP32 FFT convolutions vs FP64


@pytest.fixture(scope="module")
def mg(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg

    return mg


def _dev(x, dtype=None):
    import torch

    return torch.as_tensor(np.asarray(x), dtype=dtype or torch.float64, device="cuda:0")


def _one_receiver(w):
    """Shot s: source src[s], receiver = its first receiver (bistatic), plus a
    backscatter shot at the first source."""
    sh = w.shots
    src = np.concatenate([sh.src, sh.src[:1]]).astype(np.int32)
    rec = np.concatenate([sh.rec[sh.rec_ptr[:-1]], sh.src[:1]]).astype(np.int32)
    return shots_mod.Shots(src, np.arange(len(src) + 1, dtype=np.int64), rec)


@pytest.mark.parametrize("bc", ["abc", "neumann"])
def test_node_responses_and_projected_columns(mg, bc):
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=150, bc=bc)
    m = w.mesh
    sh = _one_receiver(w)
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, bc)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    rng = np.random.default_rng(21)
    u = rng.standard_normal((sh.n_shots, len(s))).astype(np.float32)
    mesh = mg.mesh_from_workload(w, bc=bc)
    out = mg.approx_jacobian(mesh, 1, _dev(w.eps), sh, _dev(s), dt,
                             u=_dev(u).float(), want_phi=True)
    nodes = out["nodes"]
    anc = m.ancestor(1)
    corners = aj.coarse_corners(m.cells, anc, m.n_cells[1])
    assert sorted(nodes.tolist()) == sorted(np.unique(corners).tolist())
    phi = out["phi"].cpu().numpy()
    Lp = out["Lp"].cpu().numpy()
    vol = np.bincount(anc, weights=pb.vol, minlength=m.n_cells[1])
    for k in range(sh.n_shots):
        a, r = int(sh.src[k]), int(sh.rec[k])
        ref_phi = aj.node_responses(pb, dt, s, a, r, nodes)
        assert rel_l2(phi[k], ref_phi) < TOL
        cols = aj.approx2_columns(pb, dt, s, a, r, corners, vol)
        ref_lp = oproj.project(np.repeat(u[k:k + 1].astype(np.float64), len(cols), 0), cols, dt)
        assert rel_l2(Lp[:, k, :], ref_lp) < TOL


def test_exact_at_finest_level_with_neumann_boundary(mg):
    import torch

    w = configs.tiny_2d(n_coarse=2, n_refine=1, nt=120, bc="neumann")
    m = w.mesh
    sh = _one_receiver(w)
    mesh = mg.mesh_from_workload(w, bc="neumann")
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, "neumann")
    dt = 0.5 * pb.cfl_dt()
    s = _dev(w.wavelet(dt))
    L = m.n_levels - 1
    out = mg.approx_jacobian(mesh, L, _dev(w.eps), sh, s, dt, want_phi=True)
    phi = out["phi"].cpu().numpy()
    row = {int(v): i for i, v in enumerate(out["nodes"])}
    for j in (0, 9, m.n_cells[L] - 1):
        col = sum(pb.vol[j] / 3 * phi[:, row[int(v)]] for v in m.cells[j])
        e = torch.zeros(m.n_cells[L], dtype=torch.float64, device="cuda:0")
        e[j] = 1.0
        ex = mg.jacobian_apply(mesh, L, _dev(w.eps), sh, s, dt, e).cpu().numpy()
        assert rel_l2(col, ex) < TOL


def test_host_mode_and_node_list(mg):
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=100)
    sh = _one_receiver(w)
    mesh = mg.mesh_from_workload(w)
    pb = wave.Problem(w.mesh.coords, w.mesh.cells, w.mesh.bnd, w.eps, w.bc)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    u = np.random.default_rng(2).standard_normal((sh.n_shots, len(s))).astype(np.float32)
    d = mg.approx_jacobian(mesh, 1, _dev(w.eps), sh, _dev(s), dt, u=_dev(u).float(),
                           want_phi=True)
    h = mg.approx_jacobian(mesh, 1, w.eps, sh, s, dt, u=u, want_phi=True)
    assert np.array_equal(d["nodes"], h["nodes"])
    assert np.array_equal(d["phi"].cpu().numpy(), h["phi"])
    assert np.array_equal(d["Lp"].cpu().numpy(), h["Lp"])
    # one shot per chunk (a 1-byte budget) gives the same columns
    c = mg.approx_jacobian(mesh, 1, _dev(w.eps), sh, _dev(s), dt, u=_dev(u).float(),
                           want_phi=True, mem_budget=1)
    assert rel_l2(c["phi"].cpu().numpy(), h["phi"]) < 1e-6
    assert rel_l2(c["Lp"].cpu().numpy(), h["Lp"]) < 1e-6
    # more than one receiver per shot is not supported
    with pytest.raises(Exception):
        mg.approx_jacobian(mesh, 1, _dev(w.eps), w.shots, _dev(s), dt, want_phi=True)
