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
