"""Oracle: projected (compressed) data and its Jacobian, plain FP64 numpy.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module.

Sec. II ("Projected data") compresses every trace into two numbers through
the time inner products

    <a, b>_1 = int_0^T a(t) b(t) dt,      <a, b>_2 = (1/T) int_0^T t a(t) b(t) dt,

and forms, for measurement point i, the data y^(j)_i = <u_i, u_i>_j and,
against the simulated field u0 of the current permittivity,
y0^(j)_i = <u_i, u0_i>_j.  The ratio y^(2)_i / y^(1)_i is the relative
integrated travel time of the pulse.  Because the measured u does not depend
on the parameters c, the Jacobian of the projected data is the projection of
the trace Jacobian: d/dc_l <u_i, u0_i>_j = <u_i, d u0_i/dc_l>_j.

Reading of the discretisation (the paper states the integrals only): a trace
carries one sample per leapfrog step, sample l being the field at
t_l = (l + 1) dt (the state p_{l+1}); T = nt dt; both integrals use the
right-endpoint rectangle rule over those samples,

    <a, b>_1 = sum_l dt a_l b_l,          <a, b>_2 = (1/T) sum_l dt t_l a_l b_l.

Jacobian products, with J the trace Jacobian of wave.tangent / wave.adjoint_eps:
    forward:    (Jp v)^(j)_i = <u_i, (J v)_i>_j
    transpose:  Jp^T z = J^T w  with  w_i(t_l) = dt (z^(1)_i + z^(2)_i t_l / T) u_i(t_l),
the second being the first read as a linear form in the trace perturbation.
"""
from __future__ import annotations

import numpy as np


def sample_times(dt: float, nt: int) -> np.ndarray:
    """t_l = (l + 1) dt, l = 0..nt-1: the time of sample l of a trace."""
    return (np.arange(nt, dtype=np.float64) + 1.0) * dt


def inner(a, b, dt: float, j: int) -> np.ndarray:
    """<a_i, b_i>_j for every trace i of a, b [n_traces][nt] (j = 1 or 2)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nt = a.shape[1]
    T = nt * dt
    if j == 1:
        weight = np.full(nt, dt)
    elif j == 2:
        weight = dt * sample_times(dt, nt) / T
    else:
        raise ValueError("j must be 1 or 2")
    out = np.zeros(a.shape[0])
    for i in range(a.shape[0]):          # one trace at a time, written out
        out[i] = np.sum(weight * a[i] * b[i])
    return out


def project(a, b, dt: float) -> np.ndarray:
    """[2][n_traces]: row 0 <a_i, b_i>_1, row 1 <a_i, b_i>_2."""
    return np.stack([inner(a, b, dt, 1), inner(a, b, dt, 2)])


def adjoint_weights(u, z, dt: float) -> np.ndarray:
    """Trace weights w with <w, d> = sum_{i,j} z^(j)_i <u_i, d_i>_j for every
    trace perturbation d: w_i(t_l) = dt (z^(1)_i + z^(2)_i t_l / T) u_i(t_l).
    z: [2][n_traces]."""
    u = np.asarray(u, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    nt = u.shape[1]
    T = nt * dt
    t = sample_times(dt, nt)
    w = np.zeros_like(u)
    for i in range(u.shape[0]):
        w[i] = dt * (z[0, i] + z[1, i] * t / T) * u[i]
    return w
