"""Pins of the CUDA path that need no oracle run: properties the scheme of
Sec. 2 (Eq. 5, the leapfrog of Eq. 6) fixes exactly, checked on the FP32
GPU states.

* energy: with the Neumann boundary (D = 0) and no source after step l0,
  E_{l+1/2} = 1/2 v^T M v + 1/2 p_{l+1}^T K p_l, v = (p_{l+1} - p_l)/dt, is
  constant for l >= l0 (it changes by (p_{l+1} - p_{l-1})^T s_l e / 2 per
  step); FP32 states keep it within 1e-5 relative over 2000 steps;
* reciprocity: M, K and D are symmetric, so the trace of a source at a
  recorded at b equals the trace of a source at b recorded at a.

Every node is a receiver in the energy test, so its traces are the states
p_1 .. p_nt.
"""
import numpy as np
import pytest

from helpers import oracle_problem, rel_l2
from workloads import configs, shots as shots_mod

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg

    return mg


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _states(mg, w, dt, s):
    """p_0 .. p_nt at every node for the first shot of w, from GPU traces."""
    n = w.n_nodes
    sh = shots_mod.Shots(w.shots.src[:1].copy(), np.array([0, n], np.int64),
                         np.arange(n, dtype=np.int32))
    mesh = mg.mesh_from_workload(w)
    y = mg.forward(mesh, _dev(w.eps), sh, _dev(s), dt).cpu().numpy().astype(np.float64)
    return np.concatenate([np.zeros((1, n)), y.T], axis=0)


@pytest.mark.parametrize("make", [lambda: configs.tiny_2d(n_coarse=4, n_refine=2, bc="neumann"),
                                  lambda: configs.tiny_3d(bc="neumann")],
                         ids=["tiny_2d", "tiny_3d"])
def test_energy_constant_after_source_on_gpu(mg, make):
    w = make()
    pb = oracle_problem(w)
    dt = 0.5 * pb.cfl_dt()
    nt = 2000
    s = w.wavelet(dt, nt)
    l0 = int(3.0 / w.freq / dt) + 1        # the Ricker pulse has ended by 3/f
    s[l0:] = 0.0
    P = _states(mg, w, dt, s)

    def energy(pn, pc):
        v = (pn - pc) / dt
        return 0.5 * np.sum(v * pb.m * v) + 0.5 * np.sum(pn * (pb.K @ pc))

    E = np.array([energy(P[l + 1], P[l]) for l in range(l0, nt)])
    assert E[0] > 0
    assert np.abs(E - E[0]).max() / E[0] < 1e-5


@pytest.mark.parametrize("bc", ["abc", "dirichlet", "neumann"])
def test_reciprocity_on_gpu(mg, bc):
    w = configs.tiny_2d(n_coarse=3, n_refine=2, nt=400, bc=bc)
    dt = 0.5 * oracle_problem(w).cfl_dt()
    s = w.wavelet(dt)
    interior = np.setdiff1d(np.arange(w.n_nodes), shots_mod.boundary_nodes(w.mesh))
    a, b, c = (int(x) for x in np.random.default_rng(5).choice(interior, 3, replace=False))
    # shot 0 at a records b and c, shot 1 at b records a, shot 2 at c records a
    sh = shots_mod.Shots(np.array([a, b, c], np.int32), np.array([0, 2, 3, 4], np.int64),
                         np.array([b, c, a, a], np.int32))
    mesh = mg.mesh_from_workload(w)
    y = mg.forward(mesh, _dev(w.eps), sh, _dev(s), dt).cpu().numpy()
    assert np.abs(y[0]).max() > 0
    assert rel_l2(y[2], y[0]) < 1e-5
    assert rel_l2(y[3], y[1]) < 1e-5
