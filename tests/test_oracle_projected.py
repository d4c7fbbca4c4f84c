"""Pins of the projected-data oracle (Sec. II, "Projected data").

Facts that do not come from the oracle:
* the ratio <u,u>_2 / <u,u>_1 of a pulse symmetric about t_c is t_c / T (the
  relative integrated travel time the paper reads from it), to the accuracy
  of the rectangle rule on a smooth, rapidly decaying integrand;
* <1,1>_1 = T and <1,1>_2 = T/2 + O(dt) (the continuous integrals);
* symmetry and bilinearity of both inner products;
* the Jacobian of the projected data against complex-step derivatives of
  the projected forward data (the measured traces do not depend on c);
* the dot-product test between the projected tangent and the projected
  adjoint (trace weights built from the measured traces).
"""
import math

import numpy as np

from oracle import projected, wave
from workloads import configs


def _problem(w, eps=None):
    m = w.mesh
    return wave.Problem(m.coords, m.cells, m.bnd, w.eps if eps is None else eps, w.bc)


def test_pulse_ratio_is_relative_travel_time():
    dt, nt = 1e-3, 4000
    T = nt * dt
    t = projected.sample_times(dt, nt)
    for tc, sig in ((1.3, 0.05), (2.0, 0.1), (3.1, 0.07)):
        g = np.exp(-0.5 * ((t - tc) / sig) ** 2) * np.cos(40.0 * (t - tc))
        y = projected.project(g[None], g[None], dt)
        assert math.isclose(y[1, 0] / y[0, 0], tc / T, rel_tol=1e-10)
        # <g, g>_1 = int g^2: the Gaussian-times-cos^2 integral in closed form
        exact = sig * math.sqrt(math.pi) / 2 * (1 + math.exp(-(40.0 * sig) ** 2))
        assert math.isclose(y[0, 0], exact, rel_tol=1e-10)


def test_constants_and_bilinearity():
    dt, nt = 0.01, 700
    T = nt * dt
    one = np.ones((1, nt))
    y = projected.project(one, one, dt)
    assert math.isclose(y[0, 0], T, rel_tol=1e-13)
    assert abs(y[1, 0] - T / 2) <= dt / 2 + 1e-12
    rng = np.random.default_rng(0)
    a, b, c = rng.standard_normal((3, 5, nt))
    for j in (1, 2):
        ab = projected.inner(a, b, dt, j)
        assert np.allclose(ab, projected.inner(b, a, dt, j), rtol=1e-14, atol=0)
        lhs = projected.inner(2.5 * a + c, b, dt, j)
        rhs = 2.5 * ab + projected.inner(c, b, dt, j)
        assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())
    # the second product weights late samples more: a pulse moved later has a
    # larger ratio, an early one a smaller
    assert projected.inner(one, one, dt, 2)[0] < projected.inner(one, one, dt, 1)[0]


def _setup():
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=90)
    pb = _problem(w)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    sh = w.shots
    anc = w.mesh.ancestor(1)
    nl = w.mesh.n_cells[1]
    # "measured" traces: a different permittivity (one level-1 cell changed)
    dm = np.zeros(nl)
    dm[3] = 1.5
    um = wave.forward(_problem(w, eps=w.eps + wave.prolong(dm, anc)), dt, s, sh.src,
                      sh.rec_ptr, sh.rec)
    return w, pb, dt, s, sh, anc, nl, um


def test_projected_jacobian_matches_complex_step():
    w, pb, dt, s, sh, anc, nl, um = _setup()
    h = 1e-20
    for c in (0, 7, nl - 1):
        v = np.zeros(nl)
        v[c] = 1.0
        de = wave.prolong(v, anc)
        jp = projected.project(um, wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, de), dt)
        yc = wave.forward(_problem(w, eps=w.eps + 1j * h * de), dt, s, sh.src, sh.rec_ptr,
                          sh.rec)
        cs = projected.project(um, yc.imag, dt) / h
        assert np.abs(jp - cs).max() <= 1e-12 * np.abs(cs).max()


def test_projected_dot_product():
    w, pb, dt, s, sh, anc, nl, um = _setup()
    rng = np.random.default_rng(1)
    v = rng.standard_normal(nl)
    z = rng.standard_normal((2, sh.n_traces))
    jv = projected.project(um, wave.tangent(pb, dt, s, sh.src, sh.rec_ptr, sh.rec,
                                            wave.prolong(v, anc)), dt)
    W = projected.adjoint_weights(um, z, dt)
    jtz = wave.restrict(wave.adjoint_eps(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, W), anc, nl)
    lhs, rhs = np.sum(jv * z), np.sum(v * jtz)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.linalg.norm(jv) * np.linalg.norm(z))
    # the weights are the adjoint of the projection: <w(z), d> = sum z <u, d>_j
    d = rng.standard_normal(um.shape)
    assert math.isclose(np.sum(W * d), np.sum(z * projected.project(um, d, dt)), rel_tol=1e-12)
