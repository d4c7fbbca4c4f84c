"""Pins of the approximate-Jacobian oracle (App. A.1-A.3).

Facts that do not come from the oracle:
* approx_1 (auxiliary sources at every node, Green's functions by
  reciprocity) is the exact tangent: it equals the complex-step derivative
  of the forward traces (backscatter and bistatic, absorbing and Neumann
  boundaries) to rounding;
* discrete reciprocity: the impulse response at r of a source at i equals
  the one at i of a source at r;
* approx_2 at the finest level (corners = vertices, coarse lumped mass =
  fine lumped mass) equals approx_1 without boundary damping;
* approx_2 improves as the wavelength grows and as the level gets finer
  (the coarse mass quadrature of a smoother field).
"""
import numpy as np
import pytest

from oracle import approx_jacobian as aj
from oracle import wave
from workloads import configs, shots as shots_mod


def _pb(w, bc, eps=None):
    m = w.mesh
    return wave.Problem(m.coords, m.cells, m.bnd, w.eps if eps is None else eps, bc)


@pytest.mark.parametrize("bc", ["abc", "neumann"])
@pytest.mark.parametrize("bistatic", [False, True])
def test_approx1_is_the_exact_derivative(bc, bistatic):
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=150)
    pb = _pb(w, bc)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    src = int(w.shots.src[0])
    rec = int(w.shots.rec[1]) if bistatic else src
    anc = w.mesh.ancestor(1)
    h = 1e-20
    for c in (0, 7, 20):
        de = (anc == c).astype(float)
        a1 = aj.approx1_column(pb, dt, s, src, rec, de)
        cs = wave.forward(_pb(w, bc, w.eps + 1j * h * de), dt, s, [src], [0, 1],
                          [rec])[0].imag / h
        assert np.linalg.norm(a1 - cs) <= 1e-12 * np.linalg.norm(cs)


def test_discrete_reciprocity_of_impulse_responses():
    w = configs.tiny_2d(n_coarse=2, n_refine=2, nt=120)
    pb = _pb(w, "abc")
    dt = 0.5 * pb.cfl_dt()
    a, b = int(w.shots.src[0]), int(w.shots.rec[5])
    ga = aj.greens(pb, dt, 120, a)
    gb = aj.greens(pb, dt, 120, b)
    assert np.abs(ga[b] - gb[a]).max() <= 1e-12 * np.abs(ga[b]).max()


def test_approx2_at_finest_level_equals_approx1():
    w = configs.tiny_2d(n_coarse=2, n_refine=1, nt=120)
    m = w.mesh
    pb = _pb(w, "neumann")
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    src, rec = int(w.shots.src[0]), int(w.shots.rec[2])
    L = m.n_levels - 1
    anc = m.ancestor(L)
    corners = aj.coarse_corners(m.cells, anc, m.n_cells[L])
    assert np.array_equal(np.sort(corners, 1), np.sort(m.cells, 1))
    cols = aj.approx2_columns(pb, dt, s, src, rec, corners, pb.vol)
    for c in (0, 5, m.n_cells[L] - 1):
        de = np.zeros(m.n_cells[L])
        de[c] = 1.0
        a1 = aj.approx1_column(pb, dt, s, src, rec, de)
        assert np.linalg.norm(cols[c] - a1) <= 1e-12 * np.linalg.norm(a1)


def test_approx2_improves_with_wavelength_and_level():
    w = configs.tiny_2d(n_coarse=2, n_refine=3, nt=600)
    m = w.mesh
    pb = _pb(w, "neumann")
    dt = 0.5 * pb.cfl_dt()
    src, rec = int(w.shots.src[0]), int(w.shots.rec[1])
    med = {}
    for level in (1, 2):
        anc = m.ancestor(level)
        corners = aj.coarse_corners(m.cells, anc, m.n_cells[level])
        vol = np.bincount(anc, weights=pb.vol, minlength=m.n_cells[level])
        for fac in (1.0, 0.5, 0.25):
            s = shots_mod.ricker(w.freq * fac, dt, 600)
            cols = aj.approx2_columns(pb, dt, s, src, rec, corners, vol)
            errs = []
            for c in range(0, m.n_cells[level], max(1, m.n_cells[level] // 8)):
                exact = wave.tangent(pb, dt, s, [src], [0, 1], [rec],
                                     (anc == c).astype(float))[0]
                errs.append(np.linalg.norm(cols[c] - exact) / np.linalg.norm(exact))
            med[level, fac] = np.median(errs)
    for level in (1, 2):
        assert med[level, 1.0] > med[level, 0.5] > med[level, 0.25]
    for fac in (1.0, 0.5, 0.25):
        assert med[2, fac] < med[1, fac]
    assert med[2, 0.25] < 0.1
