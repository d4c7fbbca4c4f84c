"""Projected data and its Jacobian (Sec. II, "Projected data") on the GPU,
through the C ABI, against the FP64 oracle.

* mg_project on identical FP32 inputs agrees with the oracle's inner
  products to FP64 summation-order rounding (1e-12);
* end to end (GPU traces vs oracle traces), projected data within the trace
  tolerance and projected Jacobian products within the Jacobian tolerance;
* the projected tangent and the projected adjoint pass a dot test in FP64;
* host-pointer mode returns the device-mode bits; empty and one-sample
  trace sets.
"""
import numpy as np
import pytest

from helpers import JAC_TOL, TRACE_TOL, oracle_dt, oracle_gradient, oracle_tangent, \
    oracle_traces, rel_l2
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
def case(mg):
    import torch

    w = configs.asteroid_2d(n_refine=1, S=12, nt=400)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    nl = w.mesh.n_cells[1]
    dm = np.zeros(nl)
    dm[nl // 3] = 2.0                      # "measured" data: one level-1 cell changed
    eps_m = w.eps + wave.prolong(dm, w.mesh.ancestor(1))
    u_gpu = mg.forward(mesh, _dev(eps_m), w.shots, _dev(s), dt)
    u0_gpu = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt)
    torch.cuda.synchronize()
    return w, mesh, dt, s, nl, eps_m, u_gpu, u0_gpu


def test_project_matches_oracle_on_same_inputs(mg, case):
    w, mesh, dt, s, nl, eps_m, u, u0 = case
    y = mg.project(u, u0, dt).cpu().numpy()
    ref = oproj.project(u.cpu().numpy(), u0.cpu().numpy(), dt)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    # projected data of the traces themselves; ratio = relative travel time in (0, 1)
    yy = mg.project(u, u, dt).cpu().numpy()
    assert np.all(yy[0] > 0) and np.all((yy[1] / yy[0] > 0) & (yy[1] / yy[0] < 1))


def test_projected_data_end_to_end(mg, case):
    w, mesh, dt, s, nl, eps_m, u, u0 = case
    m, sh = w.mesh, w.shots
    pb_m = wave.Problem(m.coords, m.cells, m.bnd, eps_m, w.bc)
    um_o = wave.forward(pb_m, dt, s, sh.src, sh.rec_ptr, sh.rec)
    u0_o = oracle_traces(w, dt, s, sh)
    ref = oproj.project(um_o, u0_o, dt)
    y = mg.project(u, u0, dt).cpu().numpy()
    assert rel_l2(y[0], ref[0]) < TRACE_TOL
    assert rel_l2(y[1], ref[1]) < TRACE_TOL


def test_projected_jacobian_products(mg, case):
    import torch

    w, mesh, dt, s, nl, eps_m, u, u0 = case
    rng = np.random.default_rng(7)
    v = rng.standard_normal(nl)
    z = rng.standard_normal((2, w.shots.n_traces))
    u_np = u.cpu().numpy().astype(np.float64)
    # forward product: <u, J v>_j
    jv = mg.projected_jacobian_apply(mesh, 1, _dev(w.eps), w.shots, _dev(s), dt, _dev(v), u)
    jv_ref = oproj.project(u_np, oracle_tangent(w, dt, s, w.shots, v, 1), dt)
    assert rel_l2(jv.cpu().numpy(), jv_ref) < JAC_TOL
    # transpose product: J^T w(z)
    jtz = mg.projected_jacobian_T_apply(mesh, 1, _dev(w.eps), w.shots, _dev(s), dt, _dev(z), u,
                                        ckpt_every=64)
    jtz_ref = oracle_gradient(w, dt, s, w.shots, oproj.adjoint_weights(u_np, z, dt), 1)
    assert rel_l2(jtz.cpu().numpy(), jtz_ref) < JAC_TOL
    # dot test on the GPU outputs, FP64 inner products
    lhs = float(np.sum(jv.cpu().numpy() * z))
    rhs = float(np.sum(v * jtz.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), np.linalg.norm(jv.cpu().numpy()) *
                                        np.linalg.norm(z))
    # the weights kernel against the oracle's weights on the same FP32 traces
    wts = mg.projected_weights(u, _dev(z), dt).cpu().numpy()
    wref = oproj.adjoint_weights(u_np, z, dt)
    assert np.abs(wts - wref).max() <= 2 ** -23 * np.abs(wref).max()
    torch.cuda.synchronize()


def test_host_mode_edges(mg, case):
    w, mesh, dt, s, nl, eps_m, u, u0 = case
    a, b = u.cpu().numpy(), u0.cpu().numpy()
    assert np.array_equal(mg.project(a, b, dt), mg.project(u, u0, dt).cpu().numpy())
    z = np.random.default_rng(8).standard_normal((2, a.shape[0]))
    assert np.array_equal(mg.projected_weights(a, z, dt),
                          mg.projected_weights(u, _dev(z), dt).cpu().numpy())
    empty = np.zeros((0, 10), np.float32)
    assert mg.project(empty, empty, dt).shape == (2, 0)
    one = np.full((3, 1), 2.0, np.float32)
    y1 = mg.project(one, one, dt)
    assert np.allclose(y1[0], 4.0 * dt, rtol=1e-15) and np.allclose(y1[1], 4.0 * dt, rtol=1e-15)
