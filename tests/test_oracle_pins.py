"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks a property that the discrete scheme of App. A (leapfrog,
Eqs. (leap-frog1)-(leap-frog2) with the flux eliminated, lumped mass,
first-order absorbing boundary) must satisfy exactly or to a known bound, so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them:

* assembly: the P1 stiffness on a uniform right-triangle grid is the 5-point
  stencil; K annihilates constants and, at interior nodes, linear functions;
  lumped mass / boundary weights on the square have closed forms;
* time stepping: exact discrete energy conservation (Neumann) and the exact
  discrete energy-dissipation identity of the absorbing boundary; the
  closed-form leapfrog evolution of a Dirichlet eigenmode; the straight-ray
  travel time sqrt(eps) per unit length; normal-incidence reflection of the
  absorbing boundary; mass balance of the point source;
* derivatives: tangent vs complex-step and central differences, the adjoint
  vs the complex-step derivative of every cell, the dot-product test, the
  chain rule through the nesting map; reciprocity of the Green's function.
"""
import math

import numpy as np
import pytest
from scipy.sparse.linalg import eigsh

from oracle import wave
from workloads import configs, meshes, shots as shots_mod


def _problem(w, bc=None, eps=None):
    m = w.mesh
    return wave.Problem(m.coords, m.cells, m.bnd, w.eps if eps is None else eps,
                        w.bc if bc is None else bc)


# ------------------------------------------------------------------ assembly
def test_stiffness_is_five_point_stencil_on_uniform_grid():
    m = meshes.square_mesh(4, 1)                        # 8x8 squares, h = 1/4
    pb = wave.Problem(m.coords, m.cells, m.bnd, np.ones(len(m.cells)), "neumann")
    K = pb.K.toarray()
    x, y = m.coords[:, 0], m.coords[:, 1]
    h = 0.25
    interior = np.where((np.abs(x) < 1 - 1e-9) & (np.abs(y) < 1 - 1e-9))[0]
    for i in interior:
        nb = {j: K[i, j] for j in np.nonzero(np.abs(K[i]) > 1e-14)[0]}
        assert math.isclose(nb.pop(i), 4.0, rel_tol=1e-13)
        assert len(nb) == 4
        for j, v in nb.items():
            assert math.isclose(v, -1.0, rel_tol=1e-13)
            assert math.isclose(abs(x[j] - x[i]) + abs(y[j] - y[i]), h, rel_tol=1e-12)
    # lumped mass eps*h^2 at interior nodes, boundary weight sqrt(eps)*h on edges
    eps = 2.5
    pb = wave.Problem(m.coords, m.cells, m.bnd, np.full(len(m.cells), eps), "abc")
    assert np.allclose(pb.m[interior], eps * h * h, rtol=1e-13)
    edge = np.where((np.abs(np.abs(x) - 1) < 1e-9) ^ (np.abs(np.abs(y) - 1) < 1e-9))[0]
    assert np.allclose(pb.D[edge], math.sqrt(eps) * h, rtol=1e-13)
    assert np.allclose(pb.D[interior], 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_stiffness_kernel_and_linear_exactness(dim):
    w = configs.tiny_2d(n_coarse=3, n_refine=1) if dim == 2 else configs.tiny_3d(grid=(2, 4, 2))
    m = w.mesh
    pb = _problem(w)
    n = m.coords.shape[0]
    assert np.abs(pb.K @ np.ones(n)).max() < 1e-12
    bnodes = np.unique(m.bnd.ravel())
    interior = np.setdiff1d(np.arange(n), bnodes)
    assert len(interior) > 0
    for k in range(dim):
        r = pb.K @ m.coords[:, k]
        assert np.abs(r[interior]).max() < 1e-12
    # symmetric positive semi-definite
    assert abs(pb.K - pb.K.T).max() < 1e-14
    # total lumped mass = integral of eps
    assert math.isclose(pb.m.sum(), float((w.eps * meshes.cell_measures(m)).sum()),
                        rel_tol=1e-12)


def test_cfl_bound_is_below_true_stability_limit():
    w = configs.tiny_2d(n_coarse=3, n_refine=1)
    pb = _problem(w)
    Minv = 1.0 / pb.m
    A = pb.K.multiply(np.sqrt(Minv)[:, None]).multiply(np.sqrt(Minv)[None, :])
    lam = eigsh(A.tocsc(), k=1, which="LA", return_eigenvectors=False)[0]
    assert pb.cfl_dt() <= 2.0 / math.sqrt(lam) * (1 + 1e-12)
    assert pb.cfl_dt() > 0.3 * 2.0 / math.sqrt(lam)


# -------------------------------------------------------------- time stepping
def _energy(pb, dt, p_next, p):
    v = p_next - p
    return 0.5 * np.sum(v * (pb.m[:, None] * v)) / dt ** 2 + 0.5 * np.sum(p_next * (pb.K @ p))


def test_energy_conserved_without_boundary_loss():
    w = configs.tiny_2d(n_coarse=4, n_refine=2)
    pb = _problem(w, bc="neumann")
    dt = 0.5 * pb.cfl_dt()
    x, y = w.mesh.coords[:, 0], w.mesh.coords[:, 1]
    p0 = np.exp(-((x - 0.2) ** 2 + (y + 0.1) ** 2) / 0.05)[:, None]
    nt = 2000
    _, P = wave.forward(pb, dt, np.zeros(nt), [0], [0, 1], [0], p0=p0, pm1=p0,
                        return_states=True)
    E = np.array([_energy(pb, dt, P[l + 1], P[l]) for l in range(nt + 1)])
    assert np.abs(E - E[0]).max() / E[0] < 1e-12


def test_energy_dissipation_identity_of_absorbing_boundary():
    w = configs.tiny_2d(n_coarse=4, n_refine=2)
    pb = _problem(w, bc="abc")
    dt = 0.5 * pb.cfl_dt()
    x, y = w.mesh.coords[:, 0], w.mesh.coords[:, 1]
    p0 = np.exp(-((x - 0.2) ** 2 + (y + 0.1) ** 2) / 0.05)[:, None]
    nt = 600
    _, P = wave.forward(pb, dt, np.zeros(nt), [0], [0, 1], [0], p0=p0, pm1=p0,
                        return_states=True)
    E0 = _energy(pb, dt, P[1], P[0])
    for l in range(1, nt + 1):            # P[l+1] = p_l
        dE = _energy(pb, dt, P[l + 1], P[l]) - _energy(pb, dt, P[l], P[l - 1])
        jump = P[l + 1] - P[l - 1]
        loss = -np.sum(jump * (pb.D[:, None] * jump)) / (4.0 * dt)
        assert abs(dE - loss) < 1e-12 * E0
    assert _energy(pb, dt, P[-1], P[-2]) < 0.5 * E0


@pytest.mark.parametrize("mode", [(1, 1), (3, 2), (7, 5)])
def test_dirichlet_eigenmode_closed_form(mode):
    a, b = mode
    m = meshes.square_mesh(8, 3)                    # 64x64 squares, h = 1/32
    h, eps = 2.0 / 64, 3.0
    pb = wave.Problem(m.coords, m.cells, m.bnd, np.full(len(m.cells), eps), "dirichlet")
    dt = 0.5 * pb.cfl_dt()
    x, y = m.coords[:, 0], m.coords[:, 1]
    phi = np.sin(a * math.pi * (x + 1) / 2) * np.sin(b * math.pi * (y + 1) / 2)
    lam = (4.0 / h ** 2) * (math.sin(a * math.pi * h / 4) ** 2
                           + math.sin(b * math.pi * h / 4) ** 2) / eps
    Om = 2.0 / dt * math.asin(0.5 * dt * math.sqrt(lam))
    nt = 400
    _, P = wave.forward(pb, dt, np.zeros(nt), [0], [0, 1], [0], p0=phi[:, None],
                        pm1=(math.cos(Om * dt) * phi)[:, None], return_states=True)
    for l in range(-1, nt + 1):
        assert np.abs(P[l + 1, :, 0] - math.cos(Om * l * dt) * phi).max() < 1e-11


def test_straight_ray_travel_time():
    m = meshes.square_mesh(8, 3)
    eps = 4.0
    pb = wave.Problem(m.coords, m.cells, m.bnd, np.full(len(m.cells), eps), "abc")
    dt = 0.5 * pb.cfl_dt()
    f = shots_mod.ricker_frequency(m.mean_edge_length(), ppw=10.0)
    nt = int(3.0 / dt)
    near = lambda p: int(np.argmin(np.linalg.norm(m.coords - np.asarray(p), axis=1)))
    src, r1, r2 = near((-0.5, 0.0)), near((-0.2, 0.0)), near((0.5, 0.0))
    Y = wave.forward(pb, dt, shots_mod.ricker(f, dt, nt), [src], [0, 2], [r1, r2])
    onset = lambda tr: np.argmax(np.abs(tr) > 0.01 * np.abs(tr).max()) * dt
    dist = np.linalg.norm(m.coords[r2] - m.coords[r1])
    expected = dist * math.sqrt(eps)                # c = eps^(-1/2)
    tol = max(0.02 * expected, 0.25 / f)
    assert abs(onset(Y[1]) - onset(Y[0]) - expected) < tol
    # a wrong speed (eps^(-1) or eps^0) would be far outside the tolerance
    assert tol < 0.5 * expected


def test_absorbing_boundary_normal_incidence():
    Lx, Wy, h = 4.0, 0.25, 1.0 / 32
    c, t = meshes.rectangle_level0(int(Lx / h), int(Wy / h), 0.0, Lx, 0.0, Wy)
    m = meshes.build_hierarchy(2, c, t, 0)
    right = m.bnd[np.all(np.isclose(m.coords[m.bnd][:, :, 0], Lx), axis=1)]
    x = m.coords[:, 0]
    probe = int(np.argmin(np.abs(x - 2.5) + np.abs(m.coords[:, 1] - Wy / 2)))
    ratios = {}
    for eps in (4.0, 1.5):
        for bc, bnd in (("abc", right), ("neumann", m.bnd)):
            pb = wave.Problem(m.coords, m.cells, bnd, np.full(len(m.cells), eps), bc)
            dt = 0.5 * pb.cfl_dt()
            cc = 1.0 / math.sqrt(eps)
            g = lambda s: np.exp(-((s - 1.0) / 0.15) ** 2)
            nt = int(6.0 / cc / dt)
            _, P = wave.forward(pb, dt, np.zeros(nt), [0], [0, 1], [0],
                                p0=g(x)[:, None], pm1=g(x + cc * dt)[:, None],
                                return_states=True)
            tr = P[:, probe, 0]
            tt = (np.arange(len(tr)) - 1) * dt
            inc = np.abs(tr[tt < 2.25 / cc]).max()
            ref = np.abs(tr[tt > 3.75 / cc]).max()
            ratios[(eps, bc)] = ref / inc
    for eps in (4.0, 1.5):
        assert ratios[(eps, "abc")] < 0.02
        assert ratios[(eps, "neumann")] > 0.9


def test_point_source_mass_balance():
    """With D = 0, 1^T K = 0, so the lumped mass of the field obeys
    sum m p_{l+1} - 2 sum m p_l + sum m p_{l-1} = dt^2 s_l exactly."""
    w = configs.tiny_2d(n_coarse=3, n_refine=1, nt=80)
    pb = _problem(w, bc="neumann")
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    _, P = wave.forward(pb, dt, s, w.shots.src[:1], [0, 1], [0], return_states=True)
    Q = np.einsum("i,lis->ls", pb.m, P)[:, 0]
    for l in range(len(s)):
        assert abs(Q[l + 2] - 2 * Q[l + 1] + Q[l] - dt * dt * s[l]) < 1e-13


def test_reciprocity():
    w = configs.tiny_2d(n_coarse=3, n_refine=2, nt=150)
    pb = _problem(w, bc="abc")
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    a, b = int(w.shots.src[0]), int(w.shots.src[1])
    y = wave.forward(pb, dt, s, [a, b], [0, 1, 2], [b, a])
    assert np.abs(y[0]).max() > 1e-3
    assert np.abs(y[0] - y[1]).max() < 1e-12 * np.abs(y[0]).max()


# ---------------------------------------------------------------- derivatives
@pytest.mark.parametrize("dim", [2, 3])
def test_tangent_matches_complex_step(dim):
    w = configs.tiny_2d() if dim == 2 else configs.tiny_3d()
    pb = _problem(w)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    sh = w.shots
    de = np.random.default_rng(1).standard_normal(len(w.eps))
    dy = wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, de)
    h = 1e-20
    yc = wave.forward(_problem(w, eps=w.eps + 1j * h * de), dt, s, sh.src, sh.rec_ptr, sh.rec)
    cs = yc.imag / h
    assert np.linalg.norm(dy - cs) <= 1e-12 * np.linalg.norm(cs)


def test_tangent_matches_central_differences():
    w = configs.tiny_2d()
    pb = _problem(w)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    sh = w.shots
    de = np.random.default_rng(2).standard_normal(len(w.eps))
    dy = wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, de)
    h = 1e-3
    yp = wave.forward(_problem(w, eps=w.eps + h * de), dt, s, sh.src, sh.rec_ptr, sh.rec)
    ym = wave.forward(_problem(w, eps=w.eps - h * de), dt, s, sh.src, sh.rec_ptr, sh.rec)
    fd = (yp - ym) / (2 * h)
    assert np.linalg.norm(dy - fd) <= 1e-5 * np.linalg.norm(fd)


def test_level_column_matches_central_differences_on_square_disc():
    """square_disc_2d (4225 nodes, 2000 steps), two level-1 columns: the
    oracle's J e_j within 1e-5 of its own central difference with h = 1e-3
    (the finite-difference step of the level parameters)."""
    w = configs.square_disc_2d()
    m, sh = w.mesh, w.shots
    pb = _problem(w)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    anc = m.ancestor(1)
    h = 1e-3
    for c in (17, 201):
        de = wave.prolong(np.eye(m.n_cells[1])[c], anc)
        jv = wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, de)
        yp = wave.forward(_problem(w, eps=w.eps + h * de), dt, s, sh.src, sh.rec_ptr, sh.rec)
        ym = wave.forward(_problem(w, eps=w.eps - h * de), dt, s, sh.src, sh.rec_ptr, sh.rec)
        fd = (yp - ym) / (2 * h)
        assert np.linalg.norm(jv - fd) <= 1e-5 * np.linalg.norm(fd)


@pytest.mark.parametrize("bc", ["abc", "neumann", "dirichlet"])
def test_adjoint_matches_complex_step_per_cell(bc):
    """Every entry of the gradient of <w, y> against a complex-step derivative."""
    w = configs.tiny_2d(n_coarse=2, n_refine=1, nt=60, bc=bc)
    pb = _problem(w)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    sh = w.shots
    W = np.random.default_rng(3).standard_normal((sh.n_traces, len(s)))
    g = wave.adjoint_eps(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, W)
    h = 1e-20
    ref = np.empty(len(w.eps))
    for e in range(len(w.eps)):
        eps = w.eps.astype(complex)
        eps[e] += 1j * h
        y = wave.forward(_problem(w, eps=eps), dt, s, sh.src, sh.rec_ptr, sh.rec)
        ref[e] = np.sum(W * y.imag) / h
    assert np.abs(g - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_dot_product(dim):
    w = configs.tiny_2d() if dim == 2 else configs.tiny_3d()
    pb = _problem(w)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    sh = w.shots
    rng = np.random.default_rng(4)
    v = rng.standard_normal(len(w.eps))
    W = rng.standard_normal((sh.n_traces, len(s)))
    Jv = wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, v)
    JtW = wave.adjoint_eps(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, W)
    lhs, rhs = np.sum(Jv * W), np.sum(v * JtW)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.linalg.norm(Jv) * np.linalg.norm(W))


def test_restriction_is_chain_rule_through_nesting():
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=60)
    pb = _problem(w)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    sh = w.shots
    W = np.random.default_rng(5).standard_normal((sh.n_traces, len(s)))
    anc = w.mesh.ancestor(1)
    assert np.array_equal(anc, np.arange(len(w.eps)) // 4)
    gc = wave.restrict(wave.adjoint_eps(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, W),
                       anc, w.mesh.n_cells[1])
    h = 1e-20
    for c in (0, 5, w.mesh.n_cells[1] - 1):
        v = np.zeros(w.mesh.n_cells[1])
        v[c] = 1.0
        y = wave.forward(_problem(w, eps=w.eps + 1j * h * wave.prolong(v, anc)),
                         dt, s, sh.src, sh.rec_ptr, sh.rec)
        assert math.isclose(gc[c], np.sum(W * y.imag) / h, rel_tol=1e-10)
