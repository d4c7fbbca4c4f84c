"""Uneven batches (several independent problems, one launch per step):
each instance must come out as it would alone, and as the oracle says."""
import numpy as np
import pytest

from helpers import TRACE_TOL, oracle_dt, oracle_traces, rel_l2
from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg

    return mg


def _instances(nt=300):
    spec = [(1, 8, 0.3, 0.8), (2, 37, 1.1, 1.2), (1, 128, 2.0, 1.0), (2, 200, 4.0, 0.9)]
    out = []
    for i, (lvl, S, rot, sc) in enumerate(spec):
        w = configs.asteroid_2d(n_refine=lvl, S=S, nt=nt, seed_config=5, instance=i,
                                rotation=rot, scale=sc)
        out.append(w)
    return out


def _dev(x, dt=None):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt or torch.float64, device="cuda")


def test_forward_batch_matches_single_instances(mg):
    ws = _instances()
    meshes = [mg.mesh_from_workload(w) for w in ws]
    dts = [oracle_dt(w) for w in ws]
    wavs = [w.wavelet(dt) for w, dt in zip(ws, dts)]
    ys = mg.forward_batch(meshes, [_dev(w.eps) for w in ws], [w.shots for w in ws],
                          [_dev(s) for s in wavs], dts)
    for m, w, dt, s, y in zip(meshes, ws, dts, wavs, ys):
        alone = mg.forward(m, _dev(w.eps), w.shots, _dev(s), dt)
        assert torch.equal(alone, y)
    ref = oracle_traces(ws[1], dts[1], wavs[1], ws[1].shots)
    assert rel_l2(ys[1].cpu().numpy(), ref) < TRACE_TOL
    # host pointers: same bits
    yh = mg.forward_batch(meshes, [w.eps for w in ws], [w.shots for w in ws], wavs, dts)
    for a, b in zip(ys, yh):
        assert np.array_equal(a.cpu().numpy(), b)


def test_adjoint_batch_matches_single_instances(mg):
    ws = _instances(nt=256)
    meshes = [mg.mesh_from_workload(w) for w in ws]
    dts = [oracle_dt(w) for w in ws]
    wavs = [_dev(w.wavelet(dt)) for w, dt in zip(ws, dts)]
    eps = [_dev(w.eps) for w in ws]
    rng = np.random.default_rng(11)
    W = [_dev(rng.standard_normal((w.shots.n_traces, w.nt)), torch.float32) for w in ws]
    levels = [1, 1, 0, 1]
    gs = mg.jacobian_T_apply_batch(meshes, levels, eps, [w.shots for w in ws], wavs, dts, W,
                                   ckpt_every=64)
    for m, w, lv, e, s, dt, Wi, g in zip(meshes, ws, levels, eps, wavs, dts, W, gs):
        m.set_tuning(-1, -1, 0, -1)
        alone = mg.jacobian_T_apply(m, lv, e, w.shots, s, dt, Wi, ckpt_every=64)
        assert rel_l2(g.cpu().numpy(), alone.cpu().numpy()) < 1e-6


def test_batch_rejects_repeated_handle(mg):
    from paper_1707_04605_gb300 import _lib as L

    w = configs.tiny_2d()
    m = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    with pytest.raises(L.MgError) as e:
        mg.forward_batch([m, m], [_dev(w.eps)] * 2, [w.shots] * 2, [s, s], [dt, dt])
    assert e.value.code == L.MG_ERR_ARG
