"""Full-length parity of the CUDA path with the FP64 oracle on the workloads
at their full sizes and step counts, against oracle values stored under
tests/golden/ (tests/golden/make_golden.py; tests/test_golden.py pins them
without a GPU).  The CUDA side runs every shot of the batch in the same
launches as the benchmark; the sampled shots are compared.

Tolerances: traces within 1e-4 relative L2 of the oracle after the full
step count; Jacobian columns J e_j and gradients J^T w within 1e-3; the
dot-product identity <J e_j, w> = (J^T w)_j of the GPU results (FP64
inner products) within 1e-5 of |J e_j| |w|.
"""
import gc

import numpy as np
import pytest

from helpers import JAC_TOL, TRACE_TOL, check_fingerprint, golden, rel_l2
from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg

    return mg


def _dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def test_c4_ellipsoid_3d_full_length(mg):
    """1,814,385 nodes, 10.6M tets, all 64 shots in one launch per step,
    6000 steps: shots 0 and 40 against the oracle over the whole run; shot
    40 alone on the plain one-shot path (batching invariance)."""
    d = golden("c4_ellipsoid_3d_traces.npz")
    w = configs.ellipsoid_3d()
    check_fingerprint(d, w)
    mesh = mg.mesh_from_workload(w)
    eps = _dev(w.eps)
    dt = float(d["dt"])
    assert abs(dt / (w.cfl_fraction * mg.cfl_dt(mesh, eps)) - 1) < 1e-12
    s = _dev(w.wavelet(dt))
    y = mg.forward(mesh, eps, w.shots, s, dt).cpu().numpy()
    rows = w.shots.trace_rows(d["shots"])
    ref = d["traces"].astype(np.float64)
    assert rel_l2(y[rows], ref) < TRACE_TOL
    for r in range(len(rows)):
        assert rel_l2(y[rows[r]], ref[r]) < TRACE_TOL
    y1 = mg.forward(mesh, eps, w.shots.subset([40]), s, dt, single_source=True).cpu().numpy()
    assert rel_l2(y1, y[w.shots.trace_rows([40])]) < 1e-6
    mesh.close()


def test_c3_asteroid_2d_jacobian_full_length(mg):
    """62,641 nodes, 8000 steps, all 128 shots per launch: 20 seeded
    level-1 columns J e_j, the fused forward + J v pass, and J^T w from
    checkpoints every 256 steps with weights on shots 0 and 64 only,
    against the oracle's columns and gradient; the GPU dot-product identity
    on the 20 columns with dense random weights."""
    d = golden("c3_asteroid_2d_jacobian.npz")
    w = configs.asteroid_2d()
    check_fingerprint(d, w)
    mesh = mg.mesh_from_workload(w)
    mesh.set_uniform_ell(True)
    eps = _dev(w.eps)
    dt = float(d["dt"])
    assert abs(dt / (w.cfl_fraction * mg.cfl_dt(mesh, eps)) - 1) < 1e-12
    s = _dev(w.wavelet(dt))
    level = int(d["level"])
    nl = w.mesh.n_cells[level]
    rows = w.shots.trace_rows(d["shots"])
    cols = d["columns"].astype(np.float64)
    Wd = np.random.default_rng(3022).standard_normal((w.shots.n_traces, w.nt)).astype(np.float32)
    Wd_dev = _dev(Wd, torch.float32)
    g_dense = mg.jacobian_T_apply(mesh, level, eps, w.shots, s, dt, Wd_dev,
                                  ckpt_every=256).cpu().numpy()
    worst = 0.0
    for j, c in enumerate(d["cells"]):
        v = np.zeros(nl)
        v[int(c)] = 1.0
        jv = mg.jacobian_apply(mesh, level, eps, w.shots, s, dt, _dev(v)).cpu().numpy()
        worst = max(worst, rel_l2(jv[rows], cols[j]))
        lhs = float(np.sum(jv.astype(np.float64) * Wd.astype(np.float64)))
        scale = np.linalg.norm(jv.astype(np.float64)) * np.linalg.norm(Wd.astype(np.float64))
        assert abs(lhs - g_dense[int(c)]) <= 1e-5 * scale
    assert worst < JAC_TOL
    # the fused pass: forward traces and J e_0 in one pass
    v = np.zeros(nl)
    v[int(d["cells"][0])] = 1.0
    y, jv = mg.forward_jacobian_apply(mesh, level, eps, w.shots, s, dt, _dev(v))
    assert rel_l2(y.cpu().numpy()[rows], d["traces"]) < TRACE_TOL
    assert rel_l2(jv.cpu().numpy()[rows], cols[0]) < JAC_TOL
    # J^T w with C3's memory bound (checkpoints every 256 steps, reused)
    W = np.zeros((w.shots.n_traces, w.nt), np.float32)
    W[rows] = d["weights"]
    mg.forward(mesh, eps, w.shots, s, dt, ckpt_every=256, keep_checkpoints=True)
    g = mg.jacobian_T_apply(mesh, level, eps, w.shots, s, dt, _dev(W, torch.float32),
                            ckpt_every=256, reuse_checkpoints=True).cpu().numpy()
    assert rel_l2(g, d["gradient"]) < JAC_TOL
    mesh.close()


def test_c5_uneven_batch_full_length(mg):
    """The 24 instances of uneven_batch_2d (levels 1-4, 8-256 shots, own
    eps, shots and dt), 4000 steps: the batched forward of every shot, one
    sampled shot per instance against the oracle; the batched J^T w on the
    level-1 cells with weights on that shot only (checkpoints every 100
    steps: the spacing does not change the bits, and 256 would hold about
    215 GB of segments and checkpoints across the instances)."""
    gc.collect()
    torch.cuda.empty_cache()
    d = golden("c5_uneven_batch_2d.npz")
    ws = configs.uneven_batch_2d()
    for i, w in enumerate(ws):
        assert int(d["fp_n_nodes"][i]) == w.n_nodes
        assert abs(float(d["fp_eps_sum"][i]) / w.eps.sum() - 1) < 1e-12
    meshes = [mg.mesh_from_workload(w) for w in ws]
    eps = [_dev(w.eps) for w in ws]
    dts = [float(x) for x in d["dt"]]
    wavs = [_dev(w.wavelet(dt)) for w, dt in zip(ws, dts)]
    shots = [w.shots for w in ws]
    ys = mg.forward_batch(meshes, eps, shots, wavs, dts)
    level = int(d["level"])
    Ws = []
    for i, w in enumerate(ws):
        row = w.shots.trace_rows([int(d["shot"][i])])
        y = ys[i].cpu().numpy()[row][0]
        assert rel_l2(y, d["traces"][i]) < TRACE_TOL, f"instance {i}"
        W = np.zeros((w.shots.n_traces, w.nt), np.float32)
        W[row] = d["weights"][i]
        Ws.append(_dev(W, torch.float32))
    del ys
    gs = mg.jacobian_T_apply_batch(meshes, [level] * len(ws), eps, shots, wavs, dts, Ws,
                                   ckpt_every=100)
    ptr = d["gradient_ptr"]
    for i in range(len(ws)):
        ref = d["gradient"][ptr[i]:ptr[i + 1]].astype(np.float64)
        assert rel_l2(gs[i].cpu().numpy(), ref) < JAC_TOL, f"instance {i}"
    for m in meshes:
        m.close()
