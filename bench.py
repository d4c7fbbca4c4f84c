"""Benchmark: node-source updates per second of the leapfrog wave path.

One step = one pass of the whole path over the 2D asteroid workload
(62,641 nodes, 124,416 P1 triangles, 128 backscatter shots, 8000 leapfrog
steps): the batched forward (keeping checkpoints every 256 steps), the
adjoint gradient J^T w on the 7,776 level-1 cells (w = the traces, i.e. the
gradient of 0.5 |y|^2; recomputation from the checkpoints), and one tangent
J v.  Units per step: n * S * nt for each of the three wave fields that the
method needs (forward, adjoint, tangent); the recomputation inside the
adjoint pass and the forward re-run inside the tangent pass are overhead and
are not counted.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import configs  # noqa: E402

METRIC = "node-source updates/s (forward + adjoint + tangent wave fields)"
UNIT = "node*source updates/s"
CKPT = 256
LEVEL = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nt", type=int, default=None, help="override the step count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hbm-leg", action="store_true",
                    help="skip the 3D ellipsoid forward measurement")
    ap.add_argument("--profile", action="store_true",
                    help="only the timed device steps (for profiler launch lists)")
    ap.add_argument("--tile-rows", type=int, default=-1,
                    help="rows per shared-memory tile (0 = untiled kernels)")
    ap.add_argument("--src-tile", type=int, default=-1, help="shots per staged pass")
    ap.add_argument("--chunk", type=int, default=-1, help="leapfrog steps per CUDA graph")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-inversion-leg", action="store_true",
                    help="skip the TV-reconstruction and approximate-Jacobian timings")
    ap.add_argument("--no-batch-leg", action="store_true",
                    help="skip the uneven multi-instance batch timing")
    ap.add_argument("--min-blocks", type=int, default=-1,
                    help="register cap of the forward row kernel (0 or 5)")
    ap.add_argument("--lane-vec", type=int, default=-1,
                    help="row kernels: float4 vectors of shots per lane (1, 2, 4)")
    ap.add_argument("--hbm-only", action="store_true",
                    help="only the 3D ellipsoid forward measurement")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_for_rank(rank: int, nt=None):
    # weak scaling: every rank owns a full 128-shot batch; rank r's shots sit
    # at angles offset by r/(world) of the shot spacing (a different batch)
    w = configs.asteroid_2d(nt=nt or 8000)
    if rank:
        from workloads import shots as shots_mod

        S = w.shots.n_shots
        th_off = 2 * math.pi * rank / (S * 8)
        w.shots = shots_mod.asteroid_shots(w.mesh, S, rotation=th_off)
    return w


def describe(w):
    m = w.mesh
    return (f"asteroid_2d: {m.coords.shape[0]} nodes, {m.cells.shape[0]} P1 triangles "
            f"(level 0: {m.n_cells[0]}), {w.shots.n_shots} backscatter shots, {w.nt} steps; "
            f"forward + J^T w on {m.n_cells[LEVEL]} level-{LEVEL} cells (checkpoints every "
            f"{CKPT}) + J v")


def clocks_start():
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
             "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return None


def clocks_stop(proc, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except Exception:
        proc.kill()
        return None
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or f[0] != str(gpu_index):
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, val in zip(names, f[5:9]):
            if val.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
            "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per launch of the forward step kernel, from one
# ncu capture of the same workload and launch shape (summaries in profiles/),
# with the SHA-1 of the kernel sources at capture time: a figure is reported
# only while those sources are unchanged, else the roofline's traffic is null.
KERNEL_SOURCES = ["kernels_rows.cu", "device_util.cuh", "kernels.cuh"]
TRAFFIC = {
    # (workload, batch, tile_rows, groups, min_blocks, bulk): (bytes, sha1)
    # k_step_rows<16,2,1>, --cache-control none, mean of launches 2-5 (the
    # states stay in L2; DRAM sees write-backs)
    ("asteroid_2d", 2, 0, 1, 0, 0): (11.2e6, "cbdedf17368d2819d576b09129ba7b10fd3ce055"),
    # k_step_rows<8,2,5>, one launch
    ("ellipsoid_3d", 2, 0, 1, 5, 0): (1.668e9, "cbdedf17368d2819d576b09129ba7b10fd3ce055"),
}


def sources_sha1():
    import hashlib

    h = hashlib.sha1()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1707_04605_gb300",
                        "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_for(workload, fwd):
    key = (workload, fwd["batch"], fwd["tile_rows"], fwd.get("groups", 1),
           fwd.get("min_blocks", 0), fwd.get("bulk", 0))
    hit = TRAFFIC.get(key)
    return hit[0] if hit and hit[1] == sources_sha1() else None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                return float(d[k]), "measured"
    except Exception:
        pass
    return 6800.0, "fallback"


def hbm_leg(mg, torch, dev, nt=300, args=None):
    """The 3D ellipsoid workload (1,814,385 nodes, 64 shots; each state is
    464 MB, far beyond L2): the batched forward step over `nt` leapfrog steps,
    where the step kernel is bound by HBM bandwidth."""
    w = configs.ellipsoid_3d(nt=nt)
    mesh = mg.mesh_from_workload(w)
    eps = torch.as_tensor(w.eps, dtype=torch.float64, device=dev)
    dt = w.cfl_fraction * mg.cfl_dt(mesh, eps)
    wav = torch.as_tensor(w.wavelet(dt), dtype=torch.float64, device=dev)
    if args is not None and (args.tile_rows != -1 or args.src_tile != -1 or args.lane_vec != -1):
        mesh.set_kernel_tuning("forward", args.lane_vec, args.tile_rows, args.src_tile)
        if args.min_blocks != -1:
            mesh.set_min_blocks(args.min_blocks)
    else:
        mesh.autotune(eps, w.shots, wav, dt, steps=32, level=1)
    tuning = mesh.tuning()
    mg.forward(mesh, eps, w.shots, wav, dt)            # warm-up (graphs, buffers)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    if args is not None and args.profile:
        torch.cuda.profiler.start()
    e0.record(stream)
    mg.forward(mesh, eps, w.shots, wav, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    if args is not None and args.profile:
        torch.cuda.profiler.stop()
    s = e0.elapsed_time(e1) / 1e3
    n, S = w.n_nodes, w.shots.n_shots
    info = mesh.info()
    S_pad = 64
    bytes_step = 12.0 * n * S_pad + 8.0 * info["nnz"] + 16.0 * n
    peak, kind = peaks()
    achieved = bytes_step / (s / nt) / 1e9
    mesh.close()
    return {"workload": f"ellipsoid_3d: {n} nodes, {w.mesh.cells.shape[0]} tets, {S} "
                        f"backscatter shots, {nt} steps (forward only)",
            "forward_updates_per_s": n * S * nt / s, "us_per_leapfrog_step": 1e6 * s / nt,
            "tuning": tuning["forward"],
            "roofline": {"kernel": "k_step (batched forward leapfrog step)", "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind_note(kind),
                         "algorithmic_bytes_per_launch": bytes_step,
                         "traffic": traffic_for("ellipsoid_3d", tuning["forward"])}}


def peak_kind_note(kind):
    return "of measured" if kind == "measured" else "of fallback"


def inversion_leg(mg, torch, mesh, w, eps_d, wav_d, dt, y, nt=1000, n_cg=3):
    """One outer step of the coarse-to-fine TV reconstruction (levels 0 -> 1)
    on the bench mesh over the first `nt` steps, n_cg CG iterations per
    solve, against the cost of the J and J^T products it is made of."""
    stream = torch.cuda.current_stream()
    wav = wav_d[:nt].contiguous()
    dy = torch.as_tensor(np.ascontiguousarray(y[:, :nt]), dtype=torch.float32,
                         device=eps_d.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    kw = dict(level_f=1, alpha=1.0, beta=1.0, n_outer=1, n_cg=n_cg, cg_rtol=0.0,
              ckpt_every=200)
    mg.tv_reconstruct(mesh, 0, eps_d, w.shots, wav, dt, dy, **kw)       # warm-up
    torch.cuda.synchronize()
    ev[0].record(stream)
    x, hist = mg.tv_reconstruct(mesh, 0, eps_d, w.shots, wav, dt, dy, **kw)
    ev[1].record(stream)
    v = torch.zeros(w.mesh.n_cells[1], dtype=torch.float64, device=eps_d.device)
    v[0] = 1.0
    mg.forward(mesh, eps_d, w.shots, wav, dt, ckpt_every=200, keep_checkpoints=True)
    ev[2].record(stream)
    jv = mg.jacobian_apply(mesh, 1, eps_d, w.shots, wav, dt, v)
    ev[3].record(stream)
    mg.jacobian_T_apply(mesh, 1, eps_d, w.shots, wav, dt, jv, ckpt_every=200,
                        reuse_checkpoints=True)
    ev[4].record(stream)
    torch.cuda.synchronize()
    total = ev[0].elapsed_time(ev[1]) / 1e3
    t_fwd = ev[1].elapsed_time(ev[2]) / 1e3
    t_j = ev[2].elapsed_time(ev[3]) / 1e3
    t_jt = ev[3].elapsed_time(ev[4]) / 1e3
    it = int(hist[0, 0] + hist[0, 2])
    # one forward with checkpoints; J: one per CG iteration + the fine residual;
    # J^T: one per CG iteration + the two right-hand sides
    parts = t_fwd + (it + 1) * t_j + (it + 2) * t_jt
    return {"workload": f"{w.name} levels 0->1 ({w.mesh.n_cells[0]} -> {w.mesh.n_cells[1]} "
                        f"cells), {nt} steps, 1 outer step, {n_cg} CG iterations per solve",
            "seconds": total, "cg_iterations": [int(hist[0, 0]), int(hist[0, 2])],
            "forward_J_JT_seconds": [t_fwd, t_j, t_jt],
            "seconds_per_cg_iteration": total / max(1, it),
            "overhead_vs_its_wave_solves": total / parts - 1.0}


def approx_jacobian_leg(mg, torch, mesh, w, eps_d, wav_d, dt, y, level=1, n_check=3):
    """The paper's approximate projected Jacobian (all cells of `level`, every
    shot) against exact J e_j columns: time and the relative error on a few
    cells."""
    stream = torch.cuda.current_stream()
    u = torch.as_tensor(np.ascontiguousarray(y), dtype=torch.float32, device=eps_d.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    out = mg.approx_jacobian(mesh, level, eps_d, w.shots, wav_d, dt, u=u,
                             mem_budget=16 << 30)
    ev[1].record(stream)
    torch.cuda.synchronize()
    Lp = out["Lp"]
    nl = w.mesh.n_cells[level]
    cells = np.linspace(0, nl - 1, n_check).astype(int)
    errs = []
    t_exact = 0.0
    for j in cells:
        v = torch.zeros(nl, dtype=torch.float64, device=eps_d.device)
        v[int(j)] = 1.0
        ev[2].record(stream)
        jv = mg.jacobian_apply(mesh, level, eps_d, w.shots, wav_d, dt, v)
        ev[3].record(stream)
        ex = mg.project(u, jv, dt)
        torch.cuda.synchronize()
        t_exact += ev[2].elapsed_time(ev[3]) / 1e3
        a = Lp[:, :, int(j)]
        errs.append(float(torch.linalg.norm(a - ex) / torch.linalg.norm(ex)))
    t_col = t_exact / len(cells)
    t_approx = ev[0].elapsed_time(ev[1]) / 1e3
    return {"workload": f"{w.name} level {level}: {nl} cells x {w.shots.n_shots} shots, "
                        f"{len(wav_d)} steps, {len(out['nodes'])} corner nodes",
            "seconds": t_approx, "exact_column_seconds": t_col,
            "speedup_vs_exact_columns": nl * t_col / t_approx,
            "relative_error_sampled_cells": errs}


def batch_leg(mg, torch, dev, nt=1000, ckpt=50):
    """The uneven batch: 24 asteroid instances (levels 1-4, 8-256 shots, own
    eps, shots, f and dt) advanced by one launch per step for all of them
    (forward, and J^T with its recompute and reverse steps), against the
    same instances run one after another through the single-instance calls."""
    ws = configs.uneven_batch_2d(nt=nt)
    meshes = [mg.mesh_from_workload(w) for w in ws]
    eps = [torch.as_tensor(w.eps, dtype=torch.float64, device=dev) for w in ws]
    dts = [wi.cfl_fraction * mg.cfl_dt(m, e) for wi, m, e in zip(ws, meshes, eps)]
    wavs = [torch.as_tensor(wi.wavelet(dt), dtype=torch.float64, device=dev)
            for wi, dt in zip(ws, dts)]
    shots = [wi.shots for wi in ws]
    levels = [1] * len(ws)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, out

    t_fb, ys = timed(lambda: mg.forward_batch(meshes, eps, shots, wavs, dts))
    t_fs, _ = timed(lambda: [mg.forward(m, e, sh, wv, dt)
                             for m, e, sh, wv, dt in zip(meshes, eps, shots, wavs, dts)])
    t_ab, _ = timed(lambda: mg.jacobian_T_apply_batch(meshes, levels, eps, shots, wavs, dts, ys,
                                                      ckpt_every=ckpt))
    t_as, _ = timed(lambda: [mg.jacobian_T_apply(m, 1, e, sh, wv, dt, y, ckpt_every=ckpt)
                             for m, e, sh, wv, dt, y in zip(meshes, eps, shots, wavs, dts, ys)])
    units = sum(wi.n_nodes * wi.shots.n_shots for wi in ws) * nt
    for m in meshes:
        m.close()
    nodes = [wi.n_nodes for wi in ws]
    nshots = [wi.shots.n_shots for wi in ws]
    return {"workload": f"uneven_batch_2d: {len(ws)} instances, {min(nodes)}-{max(nodes)} "
                        f"nodes, {min(nshots)}-{max(nshots)} shots, {nt} steps, "
                        f"checkpoints every {ckpt}",
            "forward_updates_per_s": {"batched": units / t_fb, "one_by_one": units / t_fs},
            "adjoint_updates_per_s": {"batched": units / t_ab, "one_by_one": units / t_as},
            "seconds": {"forward_batched": t_fb, "forward_one_by_one": t_fs,
                        "adjoint_batched": t_ab, "adjoint_one_by_one": t_as},
            "note": "adjoint seconds include the checkpointed forward and the recompute"}


def guarded(fn, *a, **k):
    """Run one of the auxiliary legs; a failure is reported inside the JSON
    line instead of ending the run."""
    try:
        return fn(*a, **k)
    except Exception as e:                      # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def cpu_baseline(w, dt, budget_s=20.0):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of
    the same workload: 2 shots, forward + tangent + adjoint over nt_s steps."""
    from oracle import wave

    m = w.mesh
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    sub = w.shots.subset([0, 1])
    nt_s = 400
    s = w.wavelet(dt, nt_s)
    t0 = time.perf_counter()
    y = wave.forward(pb, dt, s, sub.src, sub.rec_ptr, sub.rec)
    v = np.zeros(m.n_cells[LEVEL])
    v[0] = 1.0
    wave.tangent(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, wave.prolong(v, m.ancestor(LEVEL)))
    wave.adjoint_eps(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, y)
    el = time.perf_counter() - t0
    units = 3.0 * m.coords.shape[0] * sub.n_shots * nt_s
    return {"value": units / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"2 of {w.shots.n_shots} shots, {nt_s} of {w.nt} steps, forward + tangent "
                      f"+ adjoint on the full mesh ({el:.1f} s, single-threaded numpy/scipy)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload_for_rank(0, args.nt)
    from oracle import wave

    m = w.mesh
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    dt = w.cfl_fraction * pb.cfl_dt()
    sub = w.shots.subset([0])
    nt_s = 200
    s = w.wavelet(dt, nt_s)
    v = np.zeros(m.n_cells[LEVEL])
    v[0] = 1.0
    de = wave.prolong(v, m.ancestor(LEVEL))

    def step():
        y = wave.forward(pb, dt, s, sub.src, sub.rec_ptr, sub.rec)
        wave.tangent(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, de)
        wave.adjoint_eps(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, y)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    units = 3.0 * m.coords.shape[0] * sub.n_shots * nt_s * args.steps
    val = units / el
    sample = (f"1 of {w.shots.n_shots} shots, {nt_s} of {w.nt} steps per step, forward + "
              f"tangent + adjoint on the full mesh, single-threaded numpy/scipy FP64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": describe(w)},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    if args.hbm_only:
        from paper_1707_04605_gb300 import build as _b

        _b.build()
        import paper_1707_04605_gb300 as mg

        torch.cuda.set_device(dev)
        print(json.dumps(hbm_leg(mg, torch, dev, nt=args.nt or 300, args=args)))
        return 0
    torch.cuda.set_device(dev)
    from paper_1707_04605_gb300 import build as _build

    if rank == 0:
        _build.build()
    if ws > 1:
        torch.distributed.barrier()
    import paper_1707_04605_gb300 as mg
    from paper_1707_04605_gb300 import distributed as pdist

    w = workload_for_rank(rank, args.nt)
    mesh = mg.mesh_from_workload(w)
    mesh.set_tuning(args.chunk, args.lane_vec, args.tile_rows, args.src_tile)
    if args.min_blocks != -1:
        mesh.set_min_blocks(args.min_blocks)
    n, S, nt = w.n_nodes, w.shots.n_shots, w.nt
    eps_d = torch.as_tensor(w.eps, dtype=torch.float64, device=dev)
    dt = w.cfl_fraction * mg.cfl_dt(mesh, eps_d)
    wav = w.wavelet(dt)
    wav_d = torch.as_tensor(wav, dtype=torch.float64, device=dev)
    nlev = w.mesh.n_cells[LEVEL]
    v = np.zeros(nlev)
    v[np.random.default_rng(0).integers(nlev)] = 1.0
    v_d = torch.as_tensor(v, dtype=torch.float64, device=dev)
    if (args.tile_rows == -1 and args.src_tile == -1 and args.lane_vec == -1
            and not args.no_autotune):
        # launch shapes per kernel kind, timed on this problem (setup, untimed)
        mesh.autotune(eps_d, w.shots, wav_d, dt, steps=128, level=LEVEL)
    tuning = mesh.tuning()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def allreduce(g):
        if ws > 1:
            pdist.gradient_allreduce(g)
        return g

    phase_ev = {}

    def step(record=False):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        evs[0].record(stream)
        y = mg.forward(mesh, eps_d, w.shots, wav_d, dt, ckpt_every=CKPT, keep_checkpoints=True)
        evs[1].record(stream)
        g = mg.jacobian_T_apply(mesh, LEVEL, eps_d, w.shots, wav_d, dt, y, ckpt_every=CKPT,
                                reuse_checkpoints=True)
        allreduce(g)
        evs[2].record(stream)
        mg.jacobian_apply(mesh, LEVEL, eps_d, w.shots, wav_d, dt, v_d)
        evs[3].record(stream)
        if record:
            phase_ev.setdefault("ev", []).append(evs)
        return evs

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks_start() if rank == 0 else None
    launches0 = mesh.launch_count()
    times = []
    if args.profile:
        torch.cuda.profiler.start()            # profilers capture the timed steps only
    for _ in range(args.steps):
        flush.fill_(1.0)                       # evict L2 between timed steps
        evs = step(record=True)
        times.append(evs)
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.profiler.stop()
    if ws > 1:
        torch.distributed.barrier()
    launches = mesh.launch_count() - launches0
    clocks = clocks_stop(clk, dev.index) if rank == 0 else None
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "launches": int(launches),
                              "step_ms": [e[0].elapsed_time(e[3]) for e in times]}))
        return 0
    step_ms = [e[0].elapsed_time(e[3]) for e in times]
    fwd_ms = [e[0].elapsed_time(e[1]) for e in times]
    adj_ms = [e[1].elapsed_time(e[2]) for e in times]
    tan_ms = [e[2].elapsed_time(e[3]) for e in times]
    total_s = sum(step_ms) / 1e3
    if ws > 1:
        t = torch.tensor([total_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    units_per_step = 3.0 * n * S * nt
    value = units_per_step * args.steps * ws / total_s

    # end to end through the public API with host buffers (pinned), copies inside
    pin = lambda a, dt_: torch.as_tensor(np.ascontiguousarray(a), dtype=dt_).pin_memory().numpy()
    eps_h, wav_h, v_h = pin(w.eps, torch.float64), pin(wav, torch.float64), pin(v, torch.float64)

    def step_host():
        y = mg.forward(mesh, eps_h, w.shots, wav_h, dt, ckpt_every=CKPT, keep_checkpoints=True)
        g = mg.jacobian_T_apply(mesh, LEVEL, eps_h, w.shots, wav_h, dt, y, ckpt_every=CKPT,
                                reuse_checkpoints=True)
        if ws > 1:
            gt = torch.as_tensor(g, device=dev)
            allreduce(gt)
            g = gt.cpu().numpy()
        jv = mg.jacobian_apply(mesh, LEVEL, eps_h, w.shots, wav_h, dt, v_h)
        return y, g, jv

    y, g, jv = step_host()
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        y, g, jv = step_host()
    e2e_s = time.perf_counter() - t0
    R = w.shots.n_traces
    h2d = 3 * (w.eps.nbytes + wav.nbytes) + 4 * R * nt + v.nbytes
    d2h = 4 * R * nt + 8 * nlev + 4 * R * nt

    # plain single-source GPU path on the same workload (forward only, 4 shots)
    sub = w.shots.subset(range(4))
    for _ in range(2):
        mg.forward(mesh, eps_d, sub, wav_d, dt, single_source=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mg.forward(mesh, eps_d, sub, wav_d, dt, single_source=True)
    e1.record(stream)
    torch.cuda.synchronize()
    single_rate = n * 4 * nt / (e0.elapsed_time(e1) / 1e3)
    fwd_rate = n * S * nt / (statistics.mean(fwd_ms) / 1e3)

    # projected data (Sec. II): the two time inner products of every trace
    # pair and the adjoint weights of the projected Jacobian, on this step's
    # traces (device-resident, timed with CUDA events)
    yd = torch.as_tensor(np.ascontiguousarray(y), dtype=torch.float32, device=dev)
    zd = torch.ones((2, R), dtype=torch.float64, device=dev)
    proj = {}
    for name, fn, nbytes in (
            ("project", lambda: mg.project(yd, yd, dt), 8 * R * nt + 16 * R),
            ("projected_weights", lambda: mg.projected_weights(yd, zd, dt), 8 * R * nt + 16 * R)):
        for _ in range(3):
            fn()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(20):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        us = a0.elapsed_time(a1) * 1e3 / 20
        proj[name] = {"us": us, "GB_per_s": nbytes / (us * 1e-6) / 1e9,
                      "bytes_per_launch": nbytes}
    inversion = None if args.no_inversion_leg else guarded(
        inversion_leg, mg, torch, mesh, w, eps_d, wav_d, dt, y)
    approx = None if args.no_inversion_leg else guarded(
        approx_jacobian_leg, mg, torch, mesh, w, eps_d, wav_d, dt, y)
    batch = None if args.no_batch_leg or ws > 1 else guarded(batch_leg, mg, torch, dev)
    proj["note"] = (f"{R} traces x {nt} samples; FP64 accumulation; inputs L2-resident; "
                    "the projected Jacobian products cost one jacobian_apply / "
                    "jacobian_T_apply each (the forward and adjoint phases above)")

    if rank != 0:
        return 0
    # roofline of the batched forward step kernel: algorithmic bytes per launch
    info = mesh.info()
    S_pad = S
    bytes_fwd = 12.0 * n * S_pad + 8.0 * info["nnz"] + 16.0 * n
    fwd_launch_s = statistics.mean(fwd_ms) / 1e3 / nt   # includes launch gaps
    peak, peak_kind = peaks()
    achieved = bytes_fwd / fwd_launch_s / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": describe(w), "nodes": n, "shots": S, "nt": nt,
                   "parallelism": f"shots: one 128-shot batch per GPU x {ws}",
                   "tuning": tuning,
                   "l2": "flushed between timed steps (256 MB write)"},
        "phases_ms": {"forward": statistics.mean(fwd_ms), "adjoint": statistics.mean(adj_ms),
                      "tangent": statistics.mean(tan_ms)},
        "forward_updates_per_s": fwd_rate,
        "single_source_forward_updates_per_s": single_rate,
        "batched_vs_single_source": fwd_rate / single_rate,
        "roofline": {"kernel": "k_step (batched forward leapfrog step)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": traffic_for("asteroid_2d", tuning["forward"]),
                     "algorithmic_bytes_per_launch": bytes_fwd,
                     "note": "per-launch time = forward phase / nt (includes launch gaps); "
                             "state (2 x 32 MB) is L2-resident"},
        "e2e": {"value": units_per_step * e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "projected_data": proj,
        "tv_reconstruction": inversion,
        "approx_jacobian": approx,
        "uneven_batch": batch,
    }
    if not args.no_hbm_leg:
        out["hbm_workload"] = guarded(hbm_leg, mg, torch, dev)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, dt)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
