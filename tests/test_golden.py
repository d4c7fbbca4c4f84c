"""The stored oracle values of the full-length parity tests (tests/golden/,
written by tests/golden/make_golden.py from oracle/ alone), checked without
a GPU:

* the workload generators still produce the inputs the values were made
  from (fingerprints of coordinates, permittivity and shot nodes);
* the stored values are the oracle's: the first samples are recomputed
  with the oracle (causality: sample l depends on steps 0..l only);
* on asteroid_2d at full size (62,641 nodes, 8000 steps) the oracle's 20
  level-1 columns J e_j agree with its own central differences at
  h = 1e-3 (App. A.1: the auxiliary system is the derivative of the
  leapfrog), and with its J^T w through the dot-product identity
  <J e_j, w> = (J^T w)_j.
"""
import numpy as np
import pytest

from helpers import check_fingerprint, golden, rel_l2
from oracle import wave
from workloads import configs

def _problem(w):
    m = w.mesh
    return wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)


@pytest.fixture(scope="module")
def c3():
    return golden("c3_asteroid_2d_jacobian.npz")


def test_c3_inputs_and_leading_samples_are_the_oracles(c3):
    w = configs.asteroid_2d()
    check_fingerprint(c3, w)
    pb = _problem(w)
    dt = float(c3["dt"])
    assert abs(dt / (w.cfl_fraction * pb.cfl_dt()) - 1) < 1e-12
    sub = w.shots.subset(c3["shots"])
    k = 400
    y = wave.forward(pb, dt, w.wavelet(dt)[:k], sub.src, sub.rec_ptr, sub.rec)
    assert rel_l2(c3["traces"][:, :k], y) < 1e-6
    # the second stored column (its cell is reached by sample 800) over its
    # first 1000 samples
    k = 1000
    v = np.zeros(w.mesh.n_cells[int(c3["level"])])
    v[int(c3["cells"][1])] = 1.0
    de = wave.prolong(v, w.mesh.ancestor(int(c3["level"])))
    dy = wave.tangent(pb, dt, w.wavelet(dt)[:k], sub.src, sub.rec_ptr, sub.rec, de)
    assert np.linalg.norm(dy) > 0
    assert rel_l2(c3["columns"][1][:, :k], dy) < 1e-6


def test_c3_columns_match_central_differences(c3):
    """Oracle J e_j (20 seeded level-1 cells, 2 shots, 8000 steps) against
    (y(eps + h e_j) - y(eps - h e_j)) / 2h with h = 1e-3: within 1e-5."""
    cols = c3["columns"].astype(np.float64)
    fd = c3["fd_columns"].astype(np.float64)
    assert cols.shape == (20, 2, 8000)
    for j in range(cols.shape[0]):
        assert np.linalg.norm(cols[j]) > 0
        assert rel_l2(fd[j], cols[j]) < 1e-5


def test_c3_gradient_is_the_transpose_of_the_columns(c3):
    """<J e_j, w> = (J^T w)_j on the full-size workload for the stored
    weights (FP64 inner products of the stored FP32 columns)."""
    cols = c3["columns"].astype(np.float64)
    W = c3["weights"].astype(np.float64)
    g = c3["gradient"]
    for j, c in enumerate(c3["cells"]):
        lhs = float(np.sum(cols[j] * W))
        scale = np.linalg.norm(cols[j]) * np.linalg.norm(W)
        assert abs(lhs - g[int(c)]) <= 1e-6 * scale


def test_c5_inputs_and_leading_samples_are_the_oracles():
    d = golden("c5_uneven_batch_2d.npz")
    ws = configs.uneven_batch_2d()
    assert len(ws) == len(d["dt"]) == 24
    for i, w in enumerate(ws):
        assert int(d["fp_n_nodes"][i]) == w.n_nodes
        assert abs(float(d["fp_eps_sum"][i]) / w.eps.sum() - 1) < 1e-12
        assert abs(float(d["fp_coords_sum"][i]) / np.abs(w.mesh.coords).sum() - 1) < 1e-12
        assert 0 <= int(d["shot"][i]) < w.shots.n_shots
        nl = w.mesh.n_cells[int(d["level"])]
        assert d["gradient_ptr"][i + 1] - d["gradient_ptr"][i] == nl
    # one small instance recomputed over its first samples
    i = int(np.argmin(d["fp_n_nodes"]))
    w = ws[i]
    pb = _problem(w)
    dt = float(d["dt"][i])
    assert abs(dt / (w.cfl_fraction * pb.cfl_dt()) - 1) < 1e-12
    sub = w.shots.subset([int(d["shot"][i])])
    k = 600
    y = wave.forward(pb, dt, w.wavelet(dt)[:k], sub.src, sub.rec_ptr, sub.rec)
    assert rel_l2(d["traces"][i, :k], y[0]) < 1e-6


def test_c4_stored_traces_shape():
    d = golden("c4_ellipsoid_3d_traces.npz")
    assert d["traces"].shape == (2, 6000)
    assert np.isfinite(d["traces"]).all() and np.abs(d["traces"]).max() > 0
    assert int(d["fp_n_nodes"]) == 1_814_385
