"""torch.autograd over the library: gradient of a trace loss w.r.t. the
permittivity of coarse-level cells equals J^T w, the oracle's gradient, and
a central difference of the GPU forward."""
import numpy as np
import pytest

from helpers import JAC_TOL, oracle_dt, oracle_gradient, rel_l2
from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg

    return mg


def test_prolong_is_nested_injection(mg):
    w = configs.asteroid_2d(n_refine=2, S=4, nt=10)
    mesh = mg.mesh_from_workload(w)
    rng = np.random.default_rng(1)
    for level in range(w.mesh.n_levels):
        v = rng.standard_normal(w.mesh.n_cells[level])
        out = mg.api.prolong(mesh, level, torch.as_tensor(v, device="cuda"),
                             torch.as_tensor(w.eps, device="cuda")).cpu().numpy()
        assert np.array_equal(out, w.eps + v[w.mesh.ancestor(level)])


def test_autograd_gradient(mg):
    from paper_1707_04605_gb300.autograd import level_traces

    w = configs.asteroid_2d(n_refine=1, S=12, nt=300)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    dev = torch.device("cuda")
    eps0 = torch.as_tensor(w.eps, device=dev)
    wav = torch.as_tensor(s, device=dev)
    level = 1
    nlev = w.mesh.n_cells[level]
    W = torch.as_tensor(np.random.default_rng(2).standard_normal((w.shots.n_traces, w.nt)),
                        dtype=torch.float32, device=dev)
    dc = torch.zeros(nlev, dtype=torch.float64, device=dev, requires_grad=True)
    y = level_traces(dc, mesh, level, eps0, w.shots, wav, dt, ckpt_every=64)
    loss = (W.double() * y.double()).sum()
    loss.backward()
    g = dc.grad.cpu().numpy()
    gd = mg.jacobian_T_apply(mesh, level, eps0, w.shots, wav, dt, W, ckpt_every=64).cpu().numpy()
    assert np.array_equal(g, gd)
    ref = oracle_gradient(w, dt, s, w.shots, W.cpu().numpy().astype(np.float64), level)
    assert rel_l2(g, ref) < JAC_TOL
    # central difference of the GPU forward along a random direction
    v = torch.as_tensor(np.random.default_rng(3).standard_normal(nlev), device=dev)
    h = 1e-2
    lp = (W.double() * level_traces(h * v, mesh, level, eps0, w.shots, wav, dt).double()).sum()
    lm = (W.double() * level_traces(-h * v, mesh, level, eps0, w.shots, wav, dt).double()).sum()
    fd = float((lp - lm) / (2 * h))
    assert abs(fd - float(np.dot(g, v.cpu().numpy()))) <= 2e-2 * abs(fd)


def test_backward_after_a_second_forward_recomputes(mg):
    """Two differentiable forwards on one handle with the same shots, dt and
    nt but different perturbations, then the backward of the first: the
    second forward rewrote the handle's checkpoints (its generation
    changed), so the first backward recomputes its own instead of reusing
    the second's, and equals a fresh J^T w at the first perturbation."""
    from paper_1707_04605_gb300.autograd import level_traces

    w = configs.asteroid_2d(n_refine=1, S=12, nt=300)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    dev = torch.device("cuda")
    eps0 = torch.as_tensor(w.eps, device=dev)
    wav = torch.as_tensor(w.wavelet(dt), device=dev)
    level = 1
    nlev = w.mesh.n_cells[level]
    rng = np.random.default_rng(4)
    W = torch.as_tensor(rng.standard_normal((w.shots.n_traces, w.nt)), dtype=torch.float32,
                        device=dev)
    dc1 = torch.as_tensor(0.5 * rng.random(nlev), device=dev).requires_grad_(True)
    dc2 = torch.as_tensor(-0.5 * rng.random(nlev), device=dev).requires_grad_(True)
    y1 = level_traces(dc1, mesh, level, eps0, w.shots, wav, dt, ckpt_every=64)
    gen1 = mesh.checkpoint_generation()
    y2 = level_traces(dc2, mesh, level, eps0, w.shots, wav, dt, ckpt_every=64)
    assert mesh.checkpoint_generation() != gen1
    (W.double() * y1.double()).sum().backward()
    eps1 = mg.api.prolong(mesh, level, dc1.detach(), eps0)
    ref = mg.jacobian_T_apply(mesh, level, eps1, w.shots, wav, dt, W, ckpt_every=64)
    assert torch.equal(dc1.grad, ref)
    (W.double() * y2.double()).sum().backward()
    eps2 = mg.api.prolong(mesh, level, dc2.detach(), eps0)
    ref2 = mg.jacobian_T_apply(mesh, level, eps2, w.shots, wav, dt, W, ckpt_every=64)
    assert torch.equal(dc2.grad, ref2)
