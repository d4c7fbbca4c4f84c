"""Shared helpers of the parity tests: the oracle side of each comparison."""
import numpy as np

from oracle import wave

TRACE_TOL = 1e-4      # relative L2 of traces vs the FP64 oracle
JAC_TOL = 1e-3        # relative L2 of Jacobian columns / gradients


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_problem(w, bc=None):
    m = w.mesh
    return wave.Problem(m.coords, m.cells, m.bnd, w.eps, bc or w.bc)


def oracle_dt(w, pb=None) -> float:
    pb = pb or oracle_problem(w)
    return w.cfl_fraction * pb.cfl_dt()


def oracle_traces(w, dt, wavelet, shots):
    pb = oracle_problem(w)
    return wave.forward(pb, dt, wavelet, shots.src, shots.rec_ptr, shots.rec)


def oracle_tangent(w, dt, wavelet, shots, v, level):
    pb = oracle_problem(w)
    de = wave.prolong(v, w.mesh.ancestor(level))
    return wave.tangent(pb, dt, wavelet, shots.src, shots.rec_ptr, shots.rec, de)


def oracle_gradient(w, dt, wavelet, shots, W, level):
    pb = oracle_problem(w)
    g = wave.adjoint_eps(pb, dt, wavelet, shots.src, shots.rec_ptr, shots.rec, W)
    return wave.restrict(g, w.mesh.ancestor(level), w.mesh.n_cells[level])


def golden(name):
    """A file of stored oracle values under tests/golden/ (written by
    tests/golden/make_golden.py, which calls only oracle/ and workloads/)."""
    import os

    return np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name))


def check_fingerprint(d, w):
    """The workload generators still give the inputs a golden file was made
    from: node and cell counts, coordinate, permittivity and squared
    permittivity sums, shot nodes and Ricker frequency."""
    m = w.mesh
    assert int(d["fp_n_nodes"]) == m.coords.shape[0], "mesh changed since the golden file"
    assert int(d["fp_n_cells"]) == m.cells.shape[0], "mesh changed since the golden file"
    assert abs(float(d["fp_coords_sum"]) / np.abs(m.coords).sum() - 1) < 1e-12
    assert abs(float(d["fp_eps_sum"]) / w.eps.sum() - 1) < 1e-12, "permittivity changed"
    assert abs(float(d["fp_eps_sq_sum"]) / (w.eps * w.eps).sum() - 1) < 1e-12
    assert np.array_equal(d["fp_src"], w.shots.src), "shot nodes changed"
    assert np.array_equal(d["fp_rec"], w.shots.rec), "receiver nodes changed"
    assert abs(float(d["fp_freq"]) / w.freq - 1) < 1e-12
