"""TV-regularised reconstruction (Sec. II) on the GPU, through the C ABI,
against the dense FP64 oracle.

The GPU driver applies L and L^T matrix-free (FP32 wave states, FP64 CG
vectors and inner products); the oracle builds L column by column from its
tangent and solves every system directly.  The difference is the FP32
error of the Jacobian products (~1e-5 relative) amplified by the condition
number kappa of the system solved, so each comparison allows
max(1e-3, 1e-4 kappa), kappa taken from the oracle's own system: ~50 for the
Tikhonov step, growing once the weights G = 1/|Dx| enter.
"""
import numpy as np
import pytest

from helpers import oracle_dt, rel_l2
from oracle import inversion as inv
from oracle import projected as oproj
from oracle import wave
from workloads import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg

    return mg


def _dev(x, dtype=None):
    import torch

    return torch.as_tensor(np.asarray(x), dtype=dtype or torch.float64, device="cuda:0")


@pytest.fixture(scope="module")
def prob():
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=90)
    m, sh = w.mesh, w.shots
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    dt = oracle_dt(w, pb)
    s = w.wavelet(dt)
    anc1 = m.ancestor(1)
    L1 = np.stack([wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec,
                                wave.prolong(np.eye(m.n_cells[1])[c], anc1)).ravel()
                   for c in range(m.n_cells[1])], 1)
    x_true = np.zeros(m.n_cells[1])
    x_true[[3, 4, 17]] = [1.0, 1.0, -0.8]
    pm = wave.Problem(m.coords, m.cells, m.bnd, w.eps + wave.prolong(x_true, anc1), w.bc)
    um = wave.forward(pm, dt, s, sh.src, sh.rec_ptr, sh.rec)
    u0 = wave.forward(pb, dt, s, sh.src, sh.rec_ptr, sh.rec)
    dy32 = (um - u0).astype(np.float32)
    anc0 = m.ancestor(0)
    s0 = inv.shared_measure(m.coords, m.cells, anc0, m.n_cells[0])
    s1 = inv.shared_measure(m.coords, m.cells, anc1, m.n_cells[1])
    parent = inv.parent_map(m.cell_parent, m.n_cells, 0, 1)
    basis, Rc, Rf = inv.fine_basis(s1, parent, m.n_cells[0])
    return dict(w=w, dt=dt, s=s, L1=L1, um=um.astype(np.float32), dy32=dy32, s0=s0, s1=s1,
                basis=basis, Rc=Rc, Rf=Rf)


def _tol(L, D, x_prev, alpha, first):
    g = inv.weights(D @ x_prev, first)
    kappa = np.linalg.cond(L.T @ L + alpha * D.T @ (g[:, None] * D))
    return max(1e-3, 1e-4 * kappa)


def test_single_level_matches_dense_oracle(mg, prob):
    import torch

    w, dt, s = prob["w"], prob["dt"], prob["s"]
    L0 = prob["L1"] @ prob["Rc"]
    D0 = inv.regularisation_matrix(prob["s0"], 1.0)
    alpha = 1e-2 * np.linalg.norm(L0, 2) ** 2
    dy = prob["dy32"]
    ref = inv.tv_irls(L0, D0, dy.ravel().astype(np.float64), alpha, 2)
    mesh = mg.mesh_from_workload(w)
    for n_outer in (1, 2):
        x, hist = mg.tv_reconstruct(mesh, 0, _dev(w.eps), w.shots, _dev(s), dt,
                                    torch.as_tensor(dy, device="cuda:0"), alpha=alpha, beta=1.0,
                                    n_outer=n_outer, n_cg=100, cg_rtol=1e-12, ckpt_every=30)
        prev = ref[n_outer - 2] if n_outer > 1 else np.zeros(L0.shape[1])
        assert rel_l2(x.cpu().numpy(), ref[n_outer - 1]) < _tol(L0, D0, prev, alpha,
                                                                n_outer == 1)
        assert np.all(hist[:, 0] >= 1) and np.all(hist[:, 1] < 1e-6)


def test_coarse_to_fine_matches_dense_oracle(mg, prob):
    import torch

    w, dt, s = prob["w"], prob["dt"], prob["s"]
    L1 = prob["L1"]
    D0 = inv.regularisation_matrix(prob["s0"], 1.0)
    D1 = inv.regularisation_matrix(prob["s1"], 1.0)
    alpha = 1e-2 * np.linalg.norm(L1 @ prob["Rc"], 2) ** 2
    dy = prob["dy32"]
    ref = inv.coarse_to_fine(L1, D1, D0, prob["Rc"], prob["Rf"], prob["basis"],
                             dy.ravel().astype(np.float64), alpha, 2)
    mesh = mg.mesh_from_workload(w)
    dyd = torch.as_tensor(dy, device="cuda:0")
    x1, _ = mg.tv_reconstruct(mesh, 0, _dev(w.eps), w.shots, _dev(s), dt, dyd, level_f=1,
                              alpha=alpha, beta=1.0, n_outer=1, n_cg=200, cg_rtol=1e-12,
                              ckpt_every=30)
    assert rel_l2(x1.cpu().numpy(), ref[0][2]) < 1e-3
    x2, hist = mg.tv_reconstruct(mesh, 0, _dev(w.eps), w.shots, _dev(s), dt, dyd, level_f=1,
                                 alpha=alpha, beta=1.0, n_outer=2, n_cg=200, cg_rtol=1e-12,
                                 ckpt_every=30)
    # the second step's tolerance from the worse of its coarse and fine systems
    Lc, Lb, Df = L1 @ prob["Rc"], L1 @ prob["Rf"], D1 @ prob["Rf"]
    K = ref[1][3]
    gf = inv.weights(Df @ ref[0][1], False)
    kappa_f = np.linalg.cond(Lb[:, K].T @ Lb[:, K] + alpha * Df[:, K].T @ (gf[:, None] * Df[:, K]))
    tol = max(_tol(Lc, D0, ref[0][0], alpha, False), 1e-4 * kappa_f)
    assert rel_l2(x2.cpu().numpy(), ref[1][2]) < tol
    assert hist.shape == (2, 4) and np.all(hist[:, 2] >= 1)
    # host-pointer mode returns the device-mode result
    xh, _ = mg.tv_reconstruct(mesh, 0, w.eps, w.shots, s, dt, dy, level_f=1, alpha=alpha,
                              beta=1.0, n_outer=1, n_cg=200, cg_rtol=1e-12, ckpt_every=30)
    assert rel_l2(xh, x1.cpu().numpy()) < 1e-6


def test_projected_data_inversion_matches_dense_oracle(mg, prob):
    import torch

    w, dt, s = prob["w"], prob["dt"], prob["s"]
    um = prob["um"]
    L1 = prob["L1"]
    R, nt = w.shots.n_traces, len(s)
    # projected Jacobian: <u_m, J e_c>_j per level-1 cell, dense
    Lp = np.stack([oproj.project(um, L1[:, c].reshape(R, nt), dt).ravel()
                   for c in range(L1.shape[1])], 1)
    dyp = oproj.project(um, prob["dy32"], dt)            # <u, u - u0>_j
    D0 = inv.regularisation_matrix(prob["s0"], 1.0)
    Lp0 = Lp @ prob["Rc"]
    alpha = 1e-2 * np.linalg.norm(Lp0, 2) ** 2
    ref = inv.tv_irls(Lp0, D0, dyp.ravel(), alpha, 1)
    mesh = mg.mesh_from_workload(w)
    x, _ = mg.tv_reconstruct(mesh, 0, _dev(w.eps), w.shots, _dev(s), dt, _dev(dyp),
                             u=torch.as_tensor(um, device="cuda:0"), alpha=alpha, beta=1.0,
                             n_outer=1,
                             n_cg=100, cg_rtol=1e-12, ckpt_every=30)
    assert rel_l2(x.cpu().numpy(), ref[0]) < 1e-3


def _level2_jacobian(w, dt, s):
    m, sh = w.mesh, w.shots
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    anc2 = m.ancestor(2)
    return np.stack([wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec,
                                  wave.prolong(np.eye(m.n_cells[2])[c], anc2)).ravel()
                     for c in range(m.n_cells[2])], 1)


def _levels_tol(L, Ds, Ps, Rs, ref, step, alpha):
    """max(1e-3, 1e-4 kappa) over the coarse and every fine system of the
    oracle's outer step `step` (weights from the step before)."""
    first = step == 0
    xc_prev = ref[step - 1][0] if step else np.zeros(Ps[0].shape[1])
    Lc = L @ Ps[0]
    g = inv.weights(Ds[0] @ xc_prev, first)
    kappas = [np.linalg.cond(Lc.T @ Lc + alpha * Ds[0].T @ (g[:, None] * Ds[0]))]
    for i in range(1, len(Ds)):
        Lf, Df = L @ Ps[i] @ Rs[i], Ds[i] @ Rs[i]
        K = ref[step][3][i - 1]
        xf_prev = ref[step - 1][1][i - 1] if step else np.zeros(Rs[i].shape[1])
        g = inv.weights(Df @ xf_prev, first)
        kappas.append(np.linalg.cond(Lf[:, K].T @ Lf[:, K] +
                                     alpha * Df[:, K].T @ (g[:, None] * Df[:, K])))
    return max(1e-3, 1e-4 * max(kappas))


@pytest.mark.parametrize("levels,keep", [([0, 1, 2], 1.0 / 3.0), ([0, 1, 2], 1.0),
                                         ([0, 2], 1.0 / 3.0)])
def test_level_recursion_matches_dense_oracle(mg, prob, levels, keep):
    """The recursion over nested levels (tv_iteration_3) against the dense
    oracle with L on the level-2 cells.  One outer step is compared element
    by element (its systems have kappa < 1e3).  From the second step on, the
    weights 1/|D x| of cells where D x nearly vanishes make kappa 1e5-1e10,
    so the solutions themselves are not determined to any useful tolerance;
    there the data misfit ||L x - dy||, which the well-determined directions
    fix, is compared instead."""
    import torch

    w, dt, s = prob["w"], prob["dt"], prob["s"]
    m = w.mesh
    L2 = _level2_jacobian(w, dt, s)
    Ds, Ps, bases, Rs = inv.hierarchy(m.coords, m.cells, m.cell_parent, m.n_cells, levels, 1.0)
    alpha = 1e-2 * np.linalg.norm(L2 @ Ps[0], 2) ** 2
    dy = prob["dy32"]
    ref = inv.coarse_to_fine_levels(L2, Ds, Ps, bases, Rs, dy.ravel().astype(np.float64),
                                    alpha, 2, keep)
    mesh = mg.mesh_from_workload(w)
    dyd = torch.as_tensor(dy, device="cuda:0")
    dy64 = dy.ravel().astype(np.float64)
    for n_outer in (1, 2):
        x, hist = mg.tv_reconstruct_levels(mesh, levels, _dev(w.eps), w.shots, _dev(s), dt, dyd,
                                           alpha=alpha, beta=1.0, n_outer=n_outer, n_cg=300,
                                           cg_rtol=1e-12, keep_frac=keep, ckpt_every=30)
        x = x.cpu().numpy()
        assert x.shape == (m.n_cells[levels[-1]],) and np.all(np.isfinite(x))
        assert hist.shape == (n_outer, 2 * len(levels))
        assert np.all(hist[:, 0::2] >= 1) and np.all(hist[0, 1::2] < 1e-6)
        if n_outer == 1:
            tol = _levels_tol(L2, Ds, Ps, Rs, ref, 0, alpha)
            assert tol < 0.1
            assert rel_l2(x, ref[0][2]) < tol
        else:
            mis, mis_ref = (np.linalg.norm(L2 @ v - dy64) for v in (x, ref[1][2]))
            assert abs(mis - mis_ref) <= 0.05 * mis_ref


def test_level_recursion_with_two_levels_is_tv_reconstruct(mg, prob):
    """mg_tv_reconstruct_levels with {0, 1} gives mg_tv_reconstruct's bits,
    and with {1} the single-level iteration on level 1."""
    import torch

    w, dt, s = prob["w"], prob["dt"], prob["s"]
    alpha = 1e-2 * np.linalg.norm(prob["L1"] @ prob["Rc"], 2) ** 2
    dyd = torch.as_tensor(prob["dy32"], device="cuda:0")
    mesh = mg.mesh_from_workload(w)
    kw = dict(alpha=alpha, beta=1.0, n_outer=2, n_cg=100, cg_rtol=1e-12, ckpt_every=30)
    a, ha = mg.tv_reconstruct(mesh, 0, _dev(w.eps), w.shots, _dev(s), dt, dyd, level_f=1, **kw)
    b, hb = mg.tv_reconstruct_levels(mesh, [0, 1], _dev(w.eps), w.shots, _dev(s), dt, dyd, **kw)
    assert torch.equal(a, b) and np.array_equal(ha, hb)
    c, _ = mg.tv_reconstruct(mesh, 1, _dev(w.eps), w.shots, _dev(s), dt, dyd, **kw)
    d, hd = mg.tv_reconstruct_levels(mesh, [1], _dev(w.eps), w.shots, _dev(s), dt, dyd, **kw)
    assert torch.equal(c, d) and hd.shape == (2, 2)
    with pytest.raises(mg._lib.MgError):
        mg.tv_reconstruct_levels(mesh, [1, 1], _dev(w.eps), w.shots, _dev(s), dt, dyd, **kw)
