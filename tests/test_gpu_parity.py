"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated for the method: FP32 state, FP64 coefficients and
reductions): traces within 1e-4 relative L2 of the oracle after the full
step count; Jacobian columns J v and gradients J^T w within 1e-3.
"""
import numpy as np
import pytest

from helpers import (JAC_TOL, TRACE_TOL, oracle_dt, oracle_gradient, oracle_problem,
                     oracle_tangent, oracle_traces, rel_l2)
from workloads import configs, shots as shots_mod

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


# ------------------------------------------------------------------ forward
def test_cfl_matches_oracle(mg):
    for w in (configs.tiny_2d(), configs.tiny_3d(), configs.square_disc_2d()):
        mesh = mg.mesh_from_workload(w)
        pb = oracle_problem(w)
        assert abs(mg.cfl_dt(mesh, _dev(w.eps)) / pb.cfl_dt() - 1) < 1e-12
        assert abs(mg.cfl_dt(mesh, w.eps) / pb.cfl_dt() - 1) < 1e-12


@pytest.mark.parametrize("make,bc,order", [
    (configs.tiny_2d, "abc", "rcm"), (configs.tiny_2d, "neumann", "morton"),
    (configs.tiny_2d, "dirichlet", "none"), (configs.tiny_3d, "abc", "rcm"),
    (configs.tiny_3d, "neumann", "morton")])
def test_forward_tiny(mg, make, bc, order):
    w = make(bc=bc)
    mesh = mg.mesh_from_workload(w, order=order)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    y = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt).cpu().numpy()
    ref = oracle_traces(w, dt, s, w.shots)
    assert rel_l2(y, ref) < TRACE_TOL


def test_forward_square_disc_2d_full(mg):
    """4225 nodes, 1 shot x 16 receivers, 2000 steps: all traces."""
    w = configs.square_disc_2d()
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    ref = oracle_traces(w, dt, s, w.shots)
    y = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt).cpu().numpy()
    assert rel_l2(y, ref) < TRACE_TOL
    per_trace = max(rel_l2(y[r], ref[r]) for r in range(len(y)))
    assert per_trace < 10 * TRACE_TOL
    # host-pointer path (copies inside the call) gives the same bits
    yh = mg.forward(mesh, w.eps, w.shots, s, dt)
    assert np.array_equal(yh, y)
    # the plain one-shot-at-a-time path
    y1 = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt, single_source=True).cpu().numpy()
    assert rel_l2(y1, ref) < TRACE_TOL


@pytest.mark.parametrize("S,nt", [(37, 900), (200, 400), (1, 600), (6, 700)])
def test_forward_asteroid_ragged_batches(mg, S, nt):
    """Level-2 asteroid mesh (15.7k nodes): padded shot counts 64 (LPR 16),
    256 (two source tiles), 4 and 8; every trace against the oracle."""
    w = configs.asteroid_2d(n_refine=2, S=S, nt=nt)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    y = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt).cpu().numpy()
    ref = oracle_traces(w, dt, s, w.shots)
    assert rel_l2(y, ref) < TRACE_TOL


def test_forward_asteroid_2d_full_sampled(mg):
    """Full workload (62,641 nodes, 128 shots, 8000 steps, one launch per
    step over all shots): shots 0 and 77 against the oracle; batching
    invariance against the plain one-shot path."""
    w = configs.asteroid_2d()
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    y = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt).cpu().numpy()
    pick = [0, 77]
    sub = w.shots.subset(pick)
    ref = oracle_traces(w, dt, s, sub)
    rows = w.shots.trace_rows(pick)
    assert rel_l2(y[rows], ref) < TRACE_TOL
    y1 = mg.forward(mesh, _dev(w.eps), sub, _dev(s), dt, single_source=True).cpu().numpy()
    assert rel_l2(y1, y[rows]) < 1e-6


def test_forward_asteroid_2d_full_all_shots_early_samples(mg):
    """Full workload, all 128 shots: the first 250 samples of every trace
    depend only on the first 250 steps, so an oracle run of 250 steps checks
    every trace of the full 8000-step launch."""
    w = configs.asteroid_2d()
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    y = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt).cpu().numpy()
    k = 250
    ref = oracle_traces(w, dt, s[:k], w.shots)
    assert rel_l2(y[:, :k], ref) < TRACE_TOL


def test_forward_ellipsoid_3d_level2(mg):
    """3D, 226,981 nodes (two refinements), 64 shots in one launch, 600
    steps: shots 0 and 33 against the oracle."""
    w = configs.ellipsoid_3d(n_refine=2, nt=600)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    y = mg.forward(mesh, _dev(w.eps), w.shots, _dev(s), dt).cpu().numpy()
    pick = [0, 33]
    sub = w.shots.subset(pick)
    ref = oracle_traces(w, dt, s, sub)
    assert rel_l2(y[w.shots.trace_rows(pick)], ref) < TRACE_TOL


def test_jacobian_ellipsoid_3d_level1(mg):
    w = configs.ellipsoid_3d(n_refine=1, S=6, nt=160)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(w.mesh.n_cells[0])
    jv = mg.jacobian_apply(mesh, 0, _dev(w.eps), w.shots, _dev(s), dt, _dev(v)).cpu().numpy()
    assert rel_l2(jv, oracle_tangent(w, dt, s, w.shots, v, 0)) < JAC_TOL
    W = rng.standard_normal((w.shots.n_traces, len(s))).astype(np.float32)
    g = mg.jacobian_T_apply(mesh, 0, _dev(w.eps), w.shots, _dev(s), dt,
                            _dev(W, torch.float32), ckpt_every=32).cpu().numpy()
    assert rel_l2(g, oracle_gradient(w, dt, s, w.shots, W.astype(np.float64), 0)) < JAC_TOL


def test_cfl_violation_rejected(mg):
    from paper_1707_04605_gb300 import _lib as L

    w = configs.tiny_2d()
    mesh = mg.mesh_from_workload(w)
    dt = 1.01 * oracle_problem(w).cfl_dt()
    with pytest.raises(L.MgError) as e:
        mg.forward(mesh, _dev(w.eps), w.shots, _dev(w.wavelet(dt)), dt)
    assert e.value.code == L.MG_ERR_CFL


# ---------------------------------------------------------------- Jacobian
@pytest.mark.parametrize("make,bc", [(configs.tiny_2d, "abc"), (configs.tiny_2d, "dirichlet"),
                                     (configs.tiny_3d, "abc")])
def test_tangent_and_adjoint_tiny(mg, make, bc):
    w = make(bc=bc)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    rng = np.random.default_rng(0)
    level = 1
    v = rng.standard_normal(w.mesh.n_cells[level])
    W = rng.standard_normal((w.shots.n_traces, len(s)))
    jv = mg.jacobian_apply(mesh, level, _dev(w.eps), w.shots, _dev(s), dt, _dev(v)).cpu().numpy()
    assert rel_l2(jv, oracle_tangent(w, dt, s, w.shots, v, level)) < JAC_TOL
    g = mg.jacobian_T_apply(mesh, level, _dev(w.eps), w.shots, _dev(s), dt,
                            _dev(W, torch.float32), ckpt_every=16).cpu().numpy()
    ref = oracle_gradient(w, dt, s, w.shots, W.astype(np.float32).astype(np.float64), level)
    assert rel_l2(g, ref) < JAC_TOL
    # dot-product test on the GPU outputs, inner products in FP64
    lhs = float(np.sum(jv.astype(np.float64) * W.astype(np.float32)))
    rhs = float(np.sum(v * g))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1e-30)


def test_adjoint_checkpoint_spacing_and_reuse(mg):
    w = configs.asteroid_2d(n_refine=1, S=12, nt=300)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    eps = _dev(w.eps)
    W = _dev(np.random.default_rng(1).standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    g7 = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=7)
    g64 = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64)
    assert torch.equal(g7, g64)
    mg.forward(mesh, eps, w.shots, s, dt, ckpt_every=64, keep_checkpoints=True)
    gr = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64,
                             reuse_checkpoints=True)
    assert torch.equal(gr, g64)
    gh = mg.jacobian_T_apply(mesh, 1, w.eps, w.shots, w.wavelet(dt), dt,
                             W.cpu().numpy(), ckpt_every=64)
    assert np.array_equal(gh, g64.cpu().numpy())


@pytest.mark.parametrize("nt,chunk,hints", [(300, 128, 0), (301, 128, 1), (300, 0, 0),
                                            (300, 128, 1)])
def test_kept_states_give_the_checkpointed_gradient(mg, nt, chunk, hints):
    """A forward that keeps every state lets J^T w skip its recompute and J v
    read the forward field: same traces, gradient and tangent bits as the
    checkpointed and recomputing paths (even and odd nt, graphs and plain
    launches, one and two shot groups); the kept states stop applying after
    a forward that does not keep them."""
    w = configs.asteroid_2d(n_refine=1, S=12, nt=nt)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(chunk, -1, -1, -1)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    eps = _dev(w.eps)
    W = _dev(np.random.default_rng(2).standard_normal((w.shots.n_traces, nt)), torch.float32)
    y_ref = mg.forward(mesh, eps, w.shots, s, dt)
    g_ref = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64)
    mesh.set_cache_hints(hints)
    y = mg.forward(mesh, eps, w.shots, s, dt, keep_states=True)
    assert torch.equal(y, y_ref)
    n0 = mesh.launch_count()
    g = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=nt,
                            reuse_checkpoints=True)
    assert torch.equal(g, g_ref)
    assert mesh.launch_count() - n0 < nt + 64          # reverse steps only, no recompute
    # reused twice: the kept states are still there
    g2 = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=nt,
                             reuse_checkpoints=True)
    assert torch.equal(g2, g_ref)
    # the tangent reads the kept forward field: same bits as recomputing it
    v = _dev(np.random.default_rng(3).standard_normal(w.mesh.n_cells[1]))
    jv_ref = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v)
    for groups in (1, 2):
        mesh.set_shot_groups(groups)
        jv = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, reuse_states=True)
        assert torch.equal(jv, jv_ref)
    mesh.set_shot_groups(1)
    # a plain forward invalidates them; the checkpointed reuse still works
    mg.forward(mesh, eps, w.shots, s, dt, ckpt_every=64, keep_checkpoints=True)
    with pytest.raises(RuntimeError):
        mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=nt,
                            reuse_checkpoints=True)
    g3 = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64,
                             reuse_checkpoints=True)
    assert torch.equal(g3, g_ref)
    with pytest.raises(RuntimeError):
        mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, reuse_states=True)


@pytest.mark.parametrize("nt,chunk,groups,keep", [(300, 128, 1, True), (301, 128, 2, True),
                                                  (300, 0, 1, False), (300, 128, 2, False)])
def test_fused_forward_tangent_gives_the_separate_results(mg, nt, chunk, groups, keep):
    """One pass for the forward traces and J v: the bits of mg_forward and
    mg_jacobian_apply; with the history kept, J^T w runs with no forward and
    gives the checkpointed gradient's bits; host pointers give the same."""
    w = configs.asteroid_2d(n_refine=1, S=12, nt=nt)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(chunk, -1, -1, -1)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    eps = _dev(w.eps)
    rng = np.random.default_rng(8)
    v = rng.standard_normal(w.mesh.n_cells[1])
    W = _dev(rng.standard_normal((w.shots.n_traces, nt)), torch.float32)
    y_ref = mg.forward(mesh, eps, w.shots, s, dt)
    jv_ref = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, _dev(v))
    g_ref = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64)
    mesh.set_shot_groups(groups, "tangent")      # the kind the fused pass runs as
    y, jv = mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, _dev(v), keep_states=keep)
    assert torch.equal(y, y_ref)
    assert torch.equal(jv, jv_ref)
    if keep:
        n0 = mesh.launch_count()
        g = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=nt,
                                reuse_checkpoints=True)
        assert torch.equal(g, g_ref)
        assert mesh.launch_count() - n0 < nt + 64
    else:
        with pytest.raises(RuntimeError):
            mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=nt,
                                reuse_checkpoints=True)
    yh, jvh = mg.forward_jacobian_apply(mesh, 1, w.eps, w.shots, w.wavelet(dt), dt, v,
                                        keep_states=keep)
    assert np.array_equal(yh, y_ref.cpu().numpy())
    assert np.array_equal(jvh, jv_ref.cpu().numpy())


@pytest.mark.parametrize("chunk,batch,tile_rows,src_tile", [
    (0, 1, 0, 32), (0, 2, 0, 32), (128, 4, 0, 32), (64, 2, 256, 16), (128, 1, 128, 64),
    (128, 2, 64, 8), (0, 4, 512, 4), (128, 2, 128, 32), (0, 2, 64, 16)])
def test_launch_shapes_give_identical_results(mg, chunk, batch, tile_rows, src_tile):
    """Graph replay vs plain launches, gather batches, shared-memory tiles of
    several sizes (including a ragged last tile) vs the untiled kernels: the
    forward and tangent steps do the same arithmetic in the same order, so
    the same bits; the adjoint's per-row sum over shots is grouped by the
    staged pass, so it agrees to FP32 rounding."""
    w = configs.asteroid_2d(n_refine=1, S=100, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    v = _dev(np.random.default_rng(3).standard_normal(w.mesh.n_cells[1]))
    W = _dev(np.random.default_rng(4).standard_normal((w.shots.n_traces, w.nt)), torch.float32)

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64))

    ref = run()
    mesh.set_tuning(chunk, batch, tile_rows, src_tile)
    out = run()
    assert torch.equal(ref[0], out[0])
    assert torch.equal(ref[1], out[1])
    assert rel_l2(out[2].cpu().numpy(), ref[2].cpu().numpy()) < 1e-5


@pytest.mark.parametrize("groups,batch,tile_rows,src_tile", [
    (2, 2, 0, 32), (4, 1, 0, 32), (8, 4, 0, 32), (2, 1, 64, 16), (4, 1, 128, 32), (8, 1, 64, 32),
])
def test_shot_groups_give_identical_results(mg, groups, batch, tile_rows, src_tile):
    """Shot groups advanced one after another inside each graph chunk and
    checkpoint segment: every shot sees the same arithmetic as in one group,
    so forward and tangent traces carry the same bits; the adjoint's per-row
    sums over shots are grouped differently (FP32 rounding)."""
    w = configs.asteroid_2d(n_refine=1, S=100, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(64, batch, tile_rows, src_tile)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    v = _dev(np.random.default_rng(3).standard_normal(w.mesh.n_cells[1]))
    W = _dev(np.random.default_rng(4).standard_normal((w.shots.n_traces, w.nt)), torch.float32)

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64))

    ref = run()
    mesh.set_shot_groups(groups)
    assert all(mesh.tuning()[k]["groups"] == groups for k in ("forward", "tangent", "adjoint"))
    out = run()
    assert torch.equal(ref[0], out[0])
    assert torch.equal(ref[1], out[1])
    assert rel_l2(out[2].cpu().numpy(), ref[2].cpu().numpy()) < 1e-5


def test_wide_batch_row_shapes_cover_every_shot(mg):
    """300 shots pad to 384 columns, which two float4 per lane (256-shot
    source tiles) cannot divide: the row kernels fall back to a tile that
    does, so every shot is advanced and matches the oracle."""
    w = configs.asteroid_2d(n_refine=1, S=300, nt=200)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    ref = mg.forward(mesh, eps, w.shots, s, dt)
    mesh.set_tuning(-1, 2, 0, 32)
    out = mg.forward(mesh, eps, w.shots, s, dt)
    assert torch.equal(ref, out)
    picks = [0, 150, 299]
    rows = w.shots.trace_rows(picks)
    y = oracle_traces(w, dt, w.wavelet(dt), w.shots.subset(picks))
    assert rel_l2(out.cpu().numpy()[rows], y) < TRACE_TOL


@pytest.mark.parametrize("batch", [1, 2, 4])
def test_register_capped_forward_gives_identical_results(mg, batch):
    """mg_mesh_set_min_blocks(5) only changes register allocation,
    mg_mesh_set_row_sweep only which CTA advances which rows,
    mg_mesh_set_l1_streaming and mg_mesh_set_late_prefetch only cache
    policy, mg_mesh_set_wide_lanes only which lane holds which shots: same
    bits."""
    w = configs.asteroid_2d(n_refine=1, S=100, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(-1, batch, 0, 32)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    W = _dev(np.random.default_rng(4).standard_normal((w.shots.n_traces, w.nt)), torch.float32)

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64))

    ref = run()
    mesh.set_min_blocks(5)
    assert mesh.tuning()["forward"]["min_blocks"] == 5
    out = run()
    assert torch.equal(ref[0], out[0])
    assert torch.equal(ref[1], out[1])
    # consecutive row blocks per CTA (a ragged last sweep included), and
    # once-read loads without L1 allocation
    for sweep in (3, 7):
        mesh.set_row_sweep(sweep)
        out = run()
        assert torch.equal(ref[0], out[0])
        assert torch.equal(ref[1], out[1])
    mesh.set_l1_streaming(not mesh.tuning()["forward"]["stream"], "forward")
    out = run()
    assert torch.equal(ref[0], out[0])
    assert torch.equal(ref[1], out[1])
    mesh.set_l1_streaming(False, "forward")
    # prefetch of the late-loaded rows (L1, L2, and the next swept block's
    # rows and entries), with the sliced and the uniformly strided stiffness
    for uniform in (False, True):
        mesh.set_uniform_ell(uniform)
        for pf in (1, 2, 3):
            mesh.set_late_prefetch(pf, "forward")
            assert mesh.tuning()["forward"]["prefetch"] == pf
            out = run()
            assert torch.equal(ref[0], out[0])
            assert torch.equal(ref[1], out[1])
    mesh.set_late_prefetch(0, "forward")
    # two 16-byte loads per gather instead of the default wide lanes (8
    # consecutive shots per lane, one 32-byte load), swept and not
    assert mesh.tuning()["forward"]["wide"] == 1
    mesh.set_wide_lanes(False)
    for sweep in (0, 3):
        mesh.set_row_sweep(sweep)
        out = run()
        assert torch.equal(ref[0], out[0])
        assert torch.equal(ref[1], out[1])
    mesh.set_wide_lanes(True)
    # the tangent's register cap: the lockstep and fused passes keep their bits
    v = _dev(np.random.default_rng(16).standard_normal(w.mesh.n_cells[1]))
    jv = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v)
    yf, jvf = mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, keep_states=True)
    mesh.set_min_blocks(5, "tangent")
    assert mesh.tuning()["tangent"]["min_blocks"] == 5
    assert torch.equal(mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v), jv)
    yc, jvc = mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, keep_states=True)
    assert torch.equal(yc, yf) and torch.equal(jvc, jvf)
    assert torch.equal(yc, ref[0])
    # the adjoint's register caps, from checkpoints and on the kept history
    g_kept = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=w.nt,
                                 reuse_checkpoints=True)
    mesh.set_late_prefetch(2, "tangent")
    yc, jvc = mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, keep_states=True)
    assert torch.equal(yc, yf) and torch.equal(jvc, jvf)
    for cap in (5, 6):
        mesh.set_min_blocks(cap, "adjoint")
        mesh.set_late_prefetch(cap - 4, "adjoint")   # L1, then L2
        assert mesh.tuning()["adjoint"]["min_blocks"] == cap
        mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, keep_states=True)
        assert torch.equal(mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=w.nt,
                                               reuse_checkpoints=True), g_kept)
        # a J^T from its own checkpoints replaces the kept history
        assert torch.equal(mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W,
                                               ckpt_every=64), ref[1])


@pytest.mark.parametrize("S,batch,groups,chunk", [(100, 2, 1, 128), (100, 1, 2, 128),
                                                   (37, 4, 1, 0), (300, 2, 1, 64)])
def test_dependent_launch_gives_identical_results(mg, S, batch, groups, chunk):
    """Row kernels launched as programmatic dependents of the previous step
    (the default; inside CUDA graphs and in plain stream order): the forward,
    tangent and adjoint give the same bits as plain launches."""
    w = configs.asteroid_2d(n_refine=1, S=S, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(chunk, batch, 0, 32)
    mesh.set_shot_groups(groups)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    rng = np.random.default_rng(6)
    W = _dev(rng.standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    v = _dev(rng.standard_normal(w.mesh.n_cells[1]))

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64))

    mesh.set_dependent_launch(False)
    ref = run()
    mesh.set_dependent_launch(True)
    out = run()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    again = run()                                 # cached graphs replayed
    for a, b in zip(ref, again):
        assert torch.equal(a, b)


@pytest.mark.parametrize("S,batch", [(100, 2), (37, 1), (300, 2)])
def test_uniform_ell_gives_identical_results(mg, S, batch):
    """The uniformly strided stiffness copy holds the same entries in the
    same order: forward, fused forward + tangent and J^T w keep their bits;
    the 3D mesh with uneven row lengths may refuse it."""
    w = configs.asteroid_2d(n_refine=1, S=S, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(-1, batch, 0, 32)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    rng = np.random.default_rng(9)
    W = _dev(rng.standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    v = _dev(rng.standard_normal(w.mesh.n_cells[1]))

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                *mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64))

    ref = run()
    mesh.set_uniform_ell(True)
    out = run()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    mesh.set_uniform_ell(False)
    for a, b in zip(ref, run()):
        assert torch.equal(a, b)


@pytest.mark.parametrize("S,batch", [(100, 1), (100, 2), (6, 1), (300, 2), (64, 2)])
def test_bulk_copied_forward_gives_identical_results(mg, S, batch):
    """Neighbour rows staged by bulk asynchronous copies: same arithmetic in
    the same order as the row kernel, so the same bits, with graphs and
    checkpoints (the adjoint's recompute uses the forward kernel too)."""
    w = configs.asteroid_2d(n_refine=1, S=S, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(-1, batch, 0, 32)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    W = _dev(np.random.default_rng(4).standard_normal((w.shots.n_traces, w.nt)), torch.float32)

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64))

    ref = run()
    mesh.set_bulk_copies(True)
    assert mesh.tuning()["forward"]["bulk"] == 1
    out = run()
    assert mesh.device_status() == 0
    assert torch.equal(ref[0], out[0])
    assert torch.equal(ref[1], out[1])


def test_autotune_picks_valid_shapes_and_keeps_results(mg):
    w = configs.asteroid_2d(n_refine=2, S=64, nt=256)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    v = _dev(np.random.default_rng(5).standard_normal(w.mesh.n_cells[1]))
    W = _dev(np.random.default_rng(6).standard_normal((w.shots.n_traces, w.nt)), torch.float32)

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64))

    ref = run()
    t = mesh.autotune(eps, w.shots, s, dt, steps=64, level=1)
    for kind in ("forward", "tangent", "adjoint"):
        assert t[kind]["batch"] in (1, 2, 4)
        assert t[kind]["tile_rows"] in (0, 64, 128, 256)
    assert mesh.autotune(eps, w.shots, s, dt, steps=64, level=1) == t   # cached
    out = run()
    assert torch.equal(ref[0], out[0])
    assert torch.equal(ref[1], out[1])
    assert rel_l2(out[2].cpu().numpy(), ref[2].cpu().numpy()) < 1e-5


def test_twenty_jacobian_columns_square_disc_2d(mg):
    """20 seeded level-1 cells of square_disc_2d (4225 nodes, 2000 steps):
    every GPU column J e_j within the Jacobian tolerance of the oracle's."""
    w = configs.square_disc_2d()
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    level = 1
    nl = w.mesh.n_cells[level]
    cells = np.random.default_rng(20).choice(nl, size=20, replace=False)
    worst = 0.0
    for c in cells:
        v = np.zeros(nl)
        v[c] = 1.0
        jv = mg.jacobian_apply(mesh, level, _dev(w.eps), w.shots, _dev(s), dt,
                               _dev(v)).cpu().numpy()
        worst = max(worst, rel_l2(jv, oracle_tangent(w, dt, s, w.shots, v, level)))
    assert worst < JAC_TOL


def test_jacobian_square_disc_2d(mg):
    """4225 nodes, 2000 steps: a level-1 column J e_j and J^T w vs oracle."""
    w = configs.square_disc_2d()
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = w.wavelet(dt)
    level = 1
    rng = np.random.default_rng(2)
    v = np.zeros(w.mesh.n_cells[level])
    v[rng.integers(len(v))] = 1.0
    jv = mg.jacobian_apply(mesh, level, _dev(w.eps), w.shots, _dev(s), dt, _dev(v)).cpu().numpy()
    assert rel_l2(jv, oracle_tangent(w, dt, s, w.shots, v, level)) < JAC_TOL
    W = rng.standard_normal((w.shots.n_traces, len(s))).astype(np.float32)
    g = mg.jacobian_T_apply(mesh, level, _dev(w.eps), w.shots, _dev(s), dt,
                            _dev(W, torch.float32), ckpt_every=256).cpu().numpy()
    assert rel_l2(g, oracle_gradient(w, dt, s, w.shots, W.astype(np.float64), level)) < JAC_TOL


@pytest.mark.parametrize("S,batch,depth", [(100, 2, 4), (100, 1, 8), (37, 4, 4), (300, 2, 8),
                                           (6, 1, 4), (64, 2, 8)])
def test_gather_ring_gives_identical_results(mg, S, batch, depth):
    """Neighbour gathers pipelined through the shared-memory ring do the
    plain gathers' FMAs in the same order: the forward (kept history and
    checkpoints), the lockstep and fused tangents, the tangent on kept
    states and both J^T w paths carry the same bits."""
    w = configs.asteroid_2d(n_refine=1, S=S, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(-1, batch, 0, 32)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    rng = np.random.default_rng(10)
    W = _dev(rng.standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    v = _dev(rng.standard_normal(w.mesh.n_cells[1]))

    def run():
        y = mg.forward(mesh, eps, w.shots, s, dt, keep_states=True)
        gk = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=w.nt,
                                 reuse_checkpoints=True)
        jvk = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, reuse_states=True)
        jv = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v)
        yf, jvf = mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v)
        g = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64)
        return y, gk, jvk, jv, yf, jvf, g

    ref = run()
    mesh.set_gather_ring(depth)
    assert all(mesh.tuning()[k]["ring"] == depth for k in ("forward", "tangent", "adjoint"))
    out = run()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    mesh.set_gather_ring(0)
    for a, b in zip(ref, run()):
        assert torch.equal(a, b)


def test_gather_ring_too_large_is_refused(mg):
    """Two gathered states of four float4 per lane at depth 8 need more
    shared memory than a CTA has: the lockstep tangent is refused with
    MG_ERR_UNSUPPORTED while the forward with the same ring runs."""
    from paper_1707_04605_gb300 import _lib as L

    w = configs.asteroid_2d(n_refine=1, S=128, nt=40)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(0, 4, 0, 32)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    v = _dev(np.random.default_rng(11).standard_normal(w.mesh.n_cells[1]))
    ref = mg.forward(mesh, eps, w.shots, s, dt)
    mesh.set_gather_ring(8)
    assert torch.equal(mg.forward(mesh, eps, w.shots, s, dt), ref)
    with pytest.raises(L.MgError) as e:
        mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v)
    assert e.value.code == L.MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("make,kw,steps", [
    (configs.square_disc_2d, {}, 128),
    (configs.asteroid_2d, dict(n_refine=1, S=100, nt=300), 64),
    (configs.asteroid_2d, dict(n_refine=1, S=37, nt=301), 7),
    (configs.tiny_3d, {}, 1000)])
def test_persistent_forward_gives_the_graph_bits(mg, make, kw, steps):
    """Several steps per cooperative launch with grid barriers between them
    (MG_PERSISTENT): each step is the block computation of the single-step
    launches, so the traces carry the same bits; its checkpoints serve
    J^T w like those of the graph path."""
    w = make(**kw)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    ref = mg.forward(mesh, eps, w.shots, s, dt)
    mesh.set_persistent(steps)
    n0 = mesh.launch_count()
    y = mg.forward(mesh, eps, w.shots, s, dt, persistent=True)
    assert torch.equal(y, ref)
    assert mesh.launch_count() - n0 < w.nt // steps + 8
    W = _dev(np.random.default_rng(12).standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    g_ref = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64)
    y2 = mg.forward(mesh, eps, w.shots, s, dt, ckpt_every=64, keep_checkpoints=True,
                    persistent=True)
    assert torch.equal(y2, ref)
    g = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64,
                            reuse_checkpoints=True)
    assert torch.equal(g, g_ref)


def test_persistent_barrier_wait_times_out_and_reports(mg):
    """A grid barrier that waits for CTAs which never arrive (a test-only
    count beyond the grid) gives up after its cycle budget: every CTA leaves,
    mg_forward returns MG_ERR_TIMEOUT, the status word is cleared and the
    handle keeps working."""
    from paper_1707_04605_gb300 import _lib as L

    w = configs.asteroid_2d(n_refine=1, S=12, nt=40)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    ref = mg.forward(mesh, eps, w.shots, s, dt)
    mesh.set_persistent(16, wait_cycles=200_000, extra_arrivals=1)
    with pytest.raises(L.MgError) as e:
        mg.forward(mesh, eps, w.shots, s, dt, persistent=True)
    assert e.value.code == L.MG_ERR_TIMEOUT
    assert mesh.device_status() == 0
    mesh.set_persistent(16)
    assert torch.equal(mg.forward(mesh, eps, w.shots, s, dt, persistent=True), ref)
    assert torch.equal(mg.forward(mesh, eps, w.shots, s, dt), ref)


def test_unknown_and_unsupported_flags_are_refused(mg):
    from paper_1707_04605_gb300 import _lib as L

    w = configs.tiny_2d()
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    v = _dev(np.ones(w.mesh.n_cells[1]))
    W = _dev(np.ones((w.shots.n_traces, w.nt)), torch.float32)
    calls = [
        lambda f: mg.forward(mesh, eps, w.shots, s, dt, flags=f),
        lambda f: mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, flags=f),
        lambda f: mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=32, flags=f),
    ]
    for call in calls:
        for f in (0x100, 0x4000):
            with pytest.raises(L.MgError) as e:
                call(f)
            assert e.value.code == L.MG_ERR_UNSUPPORTED
    for call in calls[1:]:
        with pytest.raises(L.MgError) as e:
            call(L.MG_PERSISTENT)
        assert e.value.code == L.MG_ERR_UNSUPPORTED
    with pytest.raises(L.MgError) as e:
        mg.forward(mesh, eps, w.shots, s, dt, persistent=True, keep_states=True)
    assert e.value.code == L.MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("make,kw,rows", [
    (configs.asteroid_2d, dict(n_refine=1, S=100, nt=300), 128),
    (configs.asteroid_2d, dict(n_refine=2, S=37, nt=200), 64),
    (configs.asteroid_2d, dict(n_refine=1, S=300, nt=150), 256),
    (configs.ellipsoid_3d, dict(n_refine=1, S=64, nt=120), 128)])
def test_tma_tiled_forward_gives_identical_results(mg, make, kw, rows):
    """Row tiles staged by bulk copies (producer and consumer warps, double
    buffer) do the row kernel's FMAs in the same order: the forward traces
    and the gradient (whose recompute runs the forward kind) carry the same
    bits, with graphs and plain launches; no bounded wait runs out."""
    w = make(**kw)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    W = _dev(np.random.default_rng(13).standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    level = w.mesh.n_levels - 1 if w.mesh.n_levels < 2 else 1

    def run(flags=0):
        return (mg.forward(mesh, eps, w.shots, s, dt, flags=flags),
                mg.jacobian_T_apply(mesh, level, eps, w.shots, s, dt, W, ckpt_every=64,
                                    flags=flags))

    ref = run()
    mesh.set_tma_tiles(rows)
    assert mesh.tuning()["forward"]["tma"] == rows
    for flags in (0, mg._lib.MG_NO_GRAPH):
        out = run(flags)
        assert mesh.device_status() == 0
        assert torch.equal(ref[0], out[0])
        assert torch.equal(ref[1], out[1])


def test_tma_tiled_forward_refuses_narrow_batches(mg):
    """Fewer than 32 padded shot columns cannot form a work item."""
    from paper_1707_04605_gb300 import _lib as L

    w = configs.asteroid_2d(n_refine=1, S=6, nt=20)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tma_tiles(128)
    dt = oracle_dt(w)
    with pytest.raises(L.MgError) as e:
        mg.forward(mesh, _dev(w.eps), w.shots, _dev(w.wavelet(dt)), dt)
    assert e.value.code == L.MG_ERR_UNSUPPORTED


@pytest.mark.parametrize("S,batch", [(100, 2), (100, 1), (37, 4), (300, 2)])
def test_l1_streaming_gives_identical_results(mg, S, batch):
    """Once-read loads without L1 allocation change only cache policy: the
    forward (kept history and checkpoints), the lockstep and fused
    tangents, the tangent on kept states and both J^T w paths keep their
    bits either way."""
    w = configs.asteroid_2d(n_refine=1, S=S, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(-1, batch, 0, 32)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    rng = np.random.default_rng(14)
    W = _dev(rng.standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    v = _dev(rng.standard_normal(w.mesh.n_cells[1]))

    def run():
        y = mg.forward(mesh, eps, w.shots, s, dt, keep_states=True)
        gk = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=w.nt,
                                 reuse_checkpoints=True)
        jvk = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, reuse_states=True)
        jv = mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v)
        yf, jvf = mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, keep_states=True)
        gf = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=w.nt,
                                 reuse_checkpoints=True)
        g = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64)
        return y, gk, jvk, jv, yf, jvf, gf, g

    mesh.set_l1_streaming(False)
    ref = run()
    mesh.set_l1_streaming(True)
    assert all(mesh.tuning()[k]["stream"] == 1 for k in ("forward", "tangent", "adjoint"))
    for a, b in zip(ref, run()):
        assert torch.equal(a, b)


@pytest.mark.parametrize("nt,groups,steps", [(300, 1, 64), (301, 2, 7), (300, 2, 128)])
def test_persistent_fused_pass_and_reverse_steps_give_the_graph_bits(mg, nt, groups, steps):
    """The fused forward + tangent pass writing the kept history and the
    reverse steps on it, several steps per cooperative launch: the same
    traces, J v and J^T w bits as their graph replays."""
    w = configs.asteroid_2d(n_refine=1, S=100, nt=nt)
    mesh = mg.mesh_from_workload(w)
    mesh.set_shot_groups(groups)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    eps = _dev(w.eps)
    rng = np.random.default_rng(15)
    v = _dev(rng.standard_normal(w.mesh.n_cells[1]))
    W = _dev(rng.standard_normal((w.shots.n_traces, nt)), torch.float32)

    def run(persistent):
        y, jv = mg.forward_jacobian_apply(mesh, 1, eps, w.shots, s, dt, v, keep_states=True,
                                          persistent=persistent)
        g = mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=nt,
                                reuse_checkpoints=True, persistent=persistent)
        return y, jv, g

    ref = run(False)
    mesh.set_persistent(steps)
    for a, b in zip(ref, run(True)):
        assert torch.equal(a, b)
    # a persistent J^T w needs the kept history
    from paper_1707_04605_gb300 import _lib as L

    mg.forward(mesh, eps, w.shots, s, dt, ckpt_every=64, keep_checkpoints=True)
    with pytest.raises(L.MgError) as e:
        mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64,
                            reuse_checkpoints=True, persistent=True)
    assert e.value.code == L.MG_ERR_UNSUPPORTED


def test_tuning_setters_reject_values_they_do_not_take(mg):
    """Register caps, prefetch levels and wide lanes outside their ranges
    are refused with MG_ERR_ARG and leave the tuning unchanged."""
    from paper_1707_04605_gb300 import _lib as L

    w = configs.tiny_2d()
    mesh = mg.mesh_from_workload(w)
    lib = L.load()
    before = mesh.tuning()
    K = mesh.KINDS
    for rc in (lib.mg_mesh_set_kernel_min_blocks(mesh.handle, K["forward"], 6),
               lib.mg_mesh_set_kernel_min_blocks(mesh.handle, K["tangent"], 6),
               lib.mg_mesh_set_kernel_min_blocks(mesh.handle, K["adjoint"], 7),
               lib.mg_mesh_set_kernel_min_blocks(mesh.handle, 3, 5),
               lib.mg_mesh_set_late_prefetch(mesh.handle, K["tangent"], 3),
               lib.mg_mesh_set_late_prefetch(mesh.handle, -1, 3),
               lib.mg_mesh_set_late_prefetch(mesh.handle, K["forward"], 4),
               lib.mg_mesh_set_wide_lanes(mesh.handle, 2),
               lib.mg_mesh_set_wide_lanes(None, 1),
               lib.mg_mesh_set_chunked_ell(mesh.handle, 3),
               lib.mg_mesh_set_chunked_ell(mesh.handle, 32)):
        assert rc == L.MG_ERR_ARG
    assert mesh.tuning() == before
    assert lib.mg_mesh_set_late_prefetch(mesh.handle, K["forward"], 3) == L.MG_OK
    assert lib.mg_mesh_set_kernel_min_blocks(mesh.handle, K["adjoint"], 6) == L.MG_OK
    mesh.close()


@pytest.mark.parametrize("S", [64, 37, 200])
def test_wide_lanes_and_chunked_entries_give_identical_results(mg, S):
    """The capped forward with two float4 per lane: wide lanes (8
    consecutive shots per lane, 32-byte gathers) and the chunk-major copy of
    the entries (for each lane count a launch may use), with and without the
    row sweep, the next-block prefetch and the uniformly strided copy, carry
    the bits of the uncapped two-load kernel; J^T w (its recomputed forward
    and reverse steps) and J v (the tangent kernel) read the chunk-major
    entries too and keep theirs.  Shot counts whose stride is not a multiple of 8 run the
    two-load kernel."""
    w = configs.asteroid_2d(n_refine=1, S=S, nt=300)
    eps = _dev(w.eps)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(-1, 2, 0, 32)
    dt = oracle_dt(w)
    s = _dev(w.wavelet(dt))
    W = _dev(np.random.default_rng(5).standard_normal((w.shots.n_traces, w.nt)), torch.float32)
    v = _dev(np.random.default_rng(6).standard_normal(w.mesh.n_cells[1]))

    def run():
        return (mg.forward(mesh, eps, w.shots, s, dt),
                mg.jacobian_T_apply(mesh, 1, eps, w.shots, s, dt, W, ckpt_every=64),
                mg.jacobian_apply(mesh, 1, eps, w.shots, s, dt, v))

    ref = run()
    mesh.set_min_blocks(5)
    assert mesh.tuning()["forward"]["wide"] == 1
    for chunk in (0, 2, 4, 8, 16):
        mesh.set_chunked_ell(chunk)
        for uniform, sweep, pf in ((False, 0, 0), (True, 3, 3), (False, 5, 3)):
            mesh.set_uniform_ell(uniform)
            mesh.set_row_sweep(sweep)
            mesh.set_late_prefetch(pf, "forward")
            out = run()
            for a, b in zip(ref, out):
                assert torch.equal(a, b), (chunk, uniform, sweep, pf)
    mesh.close()
