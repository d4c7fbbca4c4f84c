"""Benchmark: node-source updates per second of the leapfrog wave path.

One step = one pass of the whole path over the 2D asteroid workload
(62,641 nodes, 124,416 P1 triangles, 128 backscatter shots, 8000 leapfrog
steps): the batched forward traces, the adjoint gradient J^T w on the 7,776
level-1 cells (w = the traces, i.e. the gradient of 0.5 |y|^2) and one
tangent J v.  Units per step: n * S * nt for each of the three wave fields
the method needs (forward, adjoint, tangent); recomputation is overhead and
is not counted.

The headline step keeps every forward state in HBM when it fits (256.6 GB:
the fused forward + tangent pass writes the history, J^T w runs on it with
no recompute); the same step with forward checkpoints every 256 steps (a
recompute per segment, a bounded memory) is timed as `c3_checkpointed`.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
With --gpus N > 1 and no launcher environment, the script re-executes itself
under torch.distributed.run with N ranks.  Prints one JSON line (rank 0).
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
    ap.add_argument("--no-pml-leg", action="store_true",
                    help="skip the split-field PML path timing")
    ap.add_argument("--min-blocks", type=int, default=-1,
                    help="register cap of the forward row kernel (0 or 5)")
    ap.add_argument("--lane-vec", type=int, default=-1,
                    help="row kernels: float4 vectors of shots per lane (1, 2, 4)")
    ap.add_argument("--dep-launch", type=int, default=-1,
                    help="row kernels as programmatic dependent launches (0 or 1)")
    ap.add_argument("--checkpoints", action="store_true",
                    help="adjoint from checkpoints every 256 steps even when HBM could "
                         "hold every forward state")
    ap.add_argument("--kept-groups", default="",
                    help="shot groups forward,adjoint,tangent of the kept-history path "
                         "(instead of timing 1, 2, 4)")
    ap.add_argument("--uniform-ell", type=int, default=-1,
                    help="uniformly strided stiffness copy for the row kernels (0 or 1)")
    ap.add_argument("--chunked-ell", type=int, default=-1,
                    help="chunk-major stiffness copy: -1 for the lanes per row of the "
                         "dominant kernel, 0 off, or a chunk (2..32)")
    ap.add_argument("--cache-hints", type=int, default=-1,
                    help="kept history: L2 evict-first on the last reads (0 or 1)")
    ap.add_argument("--hbm-only", action="store_true",
                    help="only the 3D ellipsoid forward measurement")
    ap.add_argument("--no-c3-leg", action="store_true",
                    help="skip the step with checkpoints every 256 steps")
    ap.add_argument("--tuning", default="",
                    help="JSON tuning per kernel kind (as printed in config.tuning) applied "
                         "instead of the autotuner; with --hbm-only, of the 3D forward")
    return ap.parse_args()


def apply_tuning(mesh, spec):
    """Applies a tuning dict {kind: {batch, tile_rows, src_tile, groups,
    ring, min_blocks, sweep}} (the shape of Mesh.tuning()) to a handle."""
    for kind, t in spec.items():
        if kind not in ("forward", "tangent", "adjoint"):
            continue
        mesh.set_kernel_tuning(kind, t["batch"], t["tile_rows"], t["src_tile"])
        mesh.set_shot_groups(t.get("groups", 1), kind)
        mesh.set_gather_ring(t.get("ring", 0), kind)
        if "stream" in t:
            mesh.set_l1_streaming(t["stream"], kind)
        mesh.set_min_blocks(t.get("min_blocks", 0), kind)
        mesh.set_late_prefetch(t.get("prefetch", 0), kind)
        if kind == "forward":
            mesh.set_wide_lanes(t.get("wide", 1))
            mesh.set_row_sweep(t.get("sweep", 0))
            mesh.set_tma_tiles(t.get("tma", 0))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def relaunch_or_check(args):
    """--gpus N means N ranks: without a launcher environment, re-execute
    under torch.distributed.run (one process per GPU on this node); under a
    launcher, the world size must equal N."""
    if "WORLD_SIZE" not in os.environ:
        if args.gpus <= 1:
            return
        import socket

        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
               f"--nproc-per-node={args.gpus}", "--master-addr=127.0.0.1",
               f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
        os.execv(sys.executable, cmd)
    ws = int(os.environ["WORLD_SIZE"])
    if ws != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but the launcher started {ws} ranks")


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


def describe(w, layout="checkpoints"):
    """The workload and the memory layout timed: "kept" (every forward state
    in HBM, no recompute) or "checkpoints" (every CKPT steps, recompute)."""
    m = w.mesh
    how = ("every forward state kept in HBM, J^T w without recompute" if layout == "kept" else
           f"forward checkpoints every {CKPT} steps, J^T w recomputes each segment")
    return (f"asteroid_2d: {m.coords.shape[0]} nodes, {m.cells.shape[0]} P1 triangles "
            f"(level 0: {m.n_cells[0]}), {w.shots.n_shots} backscatter shots, {w.nt} steps; "
            f"forward + J^T w on {m.n_cells[LEVEL]} level-{LEVEL} cells + J v ({how})")


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


# DRAM bytes (read + write) per leapfrog step of a roofline's kernel, from
# one ncu capture of the same workload, layout and launch shape (summaries in
# profiles/), with the SHA-1 of the kernel sources at capture time: a figure
# is reported only while those sources are unchanged, else `traffic` is null.
KERNEL_SOURCES = ["rows_common.cuh", "kernels_rows.cu", "device_util.cuh", "kernels.cuh"]
TRAFFIC = {
    # key: (workload and kernel, shape_key of the kind's tuning, uniformly
    # strided stiffness); value: (DRAM bytes per leapfrog step, all shot
    # groups; sha1 of the kernel sources).  Captures (--cache-control none,
    # steady-state launches) summarised in profiles/launch_list_asteroid_2d_bench.md
    # and profiles/forward_ellipsoid_3d_s64.md.
    # k_tangent_rows<16, 1, 5, 0>, fused forward + tangent writing the kept
    # history, register cap, chunk-major entries, two shot groups of 64
    # columns: 14.9 MB read + 25.1 MB written per launch, two launches per step
    ("asteroid_2d fused", (1, 0, 2, 5, 0, 0, 0, 0, "ellc", 16), True): (80.0e6, "5d5b071a75ce9ada4d8afad12424f573dd928a35"),
    # k_adjoint_rows<16, 2, 5, 0>, reverse step on the kept history, register
    # cap, chunk-major entries, one launch of 128 columns: 42.3 MB read +
    # 21.6 MB written
    ("asteroid_2d reverse", (2, 0, 1, 5, 0, 0, 0, 0, "ellc", 16), True): (63.9e6, "5d5b071a75ce9ada4d8afad12424f573dd928a35"),
    # k_tangent_rows<16, 1, 5, 0>, lockstep forward + tangent (J v of the
    # checkpointed step), register cap, chunk-major entries, two shot groups:
    # 14.5 MB read + 17.1 MB written per launch
    ("asteroid_2d tangent", (1, 0, 2, 5, 0, 0, 0, 0, "ellc", 16), True): (63.2e6, "5d5b071a75ce9ada4d8afad12424f573dd928a35"),
    # k_step_rows_w<8, 5>, wide lanes, register cap, 4 row blocks per CTA,
    # prefetch level 3, uniformly strided stiffness with the chunk-major copy
    # for 8 lanes per row: 1249.1 MB read + 465.9 MB written per launch
    ("ellipsoid_3d forward", (2, 0, 1, 5, 0, 0, 4, 0, "prefetch", 3, "wide", "ellc", 8), True):
        (1.715e9, "5d5b071a75ce9ada4d8afad12424f573dd928a35"),
}


def shape_key(t):
    """The launch-shape fields of a kind's tuning that change its traffic."""
    return (t["batch"], t["tile_rows"], t.get("groups", 1), t.get("min_blocks", 0),
            t.get("bulk", 0), t.get("ring", 0), t.get("sweep", 0), t.get("stream", 0)) + (
        (t["tma"],) if t.get("tma", 0) else ()) + (
        ("prefetch", t["prefetch"]) if t.get("prefetch", 0) else ()) + (
        ("wide",) if t.get("wide", 0) else ()) + (
        ("ellc", t["ellc"]) if t.get("ellc", 0) else ())


def sources_sha1():
    import hashlib

    h = hashlib.sha1()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1707_04605_gb300",
                        "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def lanes_per_row(cols, nv):
    """Lanes per row of a row-kernel launch over `cols` shot columns with
    `nv` float4 per lane (the library's rule for its launch shapes)."""
    while True:
        lpr = min(32, cols // (4 * nv))
        if nv == 1 or (lpr >= 1 and lpr & (lpr - 1) == 0 and cols % (4 * nv * lpr) == 0):
            return lpr
        nv >>= 1


def set_chunked(mesh, tuning, cols, arg, kind):
    """Chunk-major stiffness entries for the lanes per row of `kind`'s row
    kernel (arg -1), of `arg` lanes (> 0) or none (0); records in every
    kind's tuning the chunk its launches use (ellc, 0 when they use the
    column layout)."""
    t = tuning[kind]
    chunk = arg
    if arg == -1:
        chunk = 0
        if t["tile_rows"] == 0:
            lpr = lanes_per_row(cols // t.get("groups", 1), t["batch"])
            chunk = lpr if 2 <= lpr <= 16 and lpr & (lpr - 1) == 0 else 0
    mesh.set_chunked_ell(chunk)
    mark_chunk(tuning, cols, chunk)
    return chunk


def mark_chunk(tuning, cols, chunk):
    """Records in each kind's tuning (a dict of Mesh.tuning()'s shape, or
    one kind's dict) the entry chunk its row-kernel launches use."""
    kinds = [tuning[k] for k in ("forward", "tangent", "adjoint") if k in tuning] \
        if "forward" in tuning else [tuning]
    for tk in kinds:
        lpr = lanes_per_row(cols // tk.get("groups", 1), tk["batch"])
        tk["ellc"] = chunk if chunk and tk["tile_rows"] == 0 and lpr == chunk else 0


def traffic_for(kernel, tuning, uniform=False):
    hit = TRAFFIC.get((kernel, shape_key(tuning), bool(uniform)))
    return hit[0] if hit and hit[1] == sources_sha1() else None


L2_BOUND = "latency (L2-resident)"    # the asteroid_2d kernels (ncu: DRAM ~1/4 of peak)


def roofline(kernel, algorithmic, seconds_per_step, traffic, peak, peak_kind, limiter, note,
             bound="hbm"):
    """Roofline of a kernel against the HBM copy rate: algorithmic bytes per
    leapfrog step over its time per step; with ncu DRAM bytes (`traffic`)
    also the DRAM fraction actually moved and the ratio of moved to
    algorithmic bytes.  `bound` names what limits the kernel per its
    profile: "hbm" where DRAM moves about the algorithmic bytes, else e.g.
    "latency (L2-resident)" (the fraction is then algorithmic-effective)."""
    achieved = algorithmic / seconds_per_step / 1e9
    out = {"kernel": kernel, "bound": bound, "denominator": "hbm", "achieved": achieved,
           "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
           "algorithmic_bytes_per_launch": algorithmic,
           "dram_frac": None if traffic is None else traffic / seconds_per_step / 1e9 / peak,
           "traffic_ratio": None if traffic is None else traffic / algorithmic,
           "limiter": limiter, "note": note}
    return out


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
    464 MB, far beyond L2): the batched forward step over `nt` of its 6000
    leapfrog steps, where the step kernel is bound by HBM bandwidth."""
    w = configs.ellipsoid_3d(nt=nt)
    mesh = mg.mesh_from_workload(w)
    eps = torch.as_tensor(w.eps, dtype=torch.float64, device=dev)
    dt = w.cfl_fraction * mg.cfl_dt(mesh, eps)
    wav = torch.as_tensor(w.wavelet(dt), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run_ms(reps=3):
        best = None
        for _ in range(reps):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            mg.forward(mesh, eps, w.shots, wav, dt)
            a1.record(stream)
            torch.cuda.synchronize()
            ms = a0.elapsed_time(a1)
            best = ms if best is None else min(best, ms)
        return best

    uniform = False
    if args is not None and args.tuning:
        t = json.loads(args.tuning)
        apply_tuning(mesh, {"forward": t})
        uniform = bool(t.get("uniform", 0))
        mesh.set_uniform_ell(uniform)
    elif args is not None and (args.tile_rows != -1 or args.src_tile != -1 or args.lane_vec != -1):
        mesh.set_kernel_tuning("forward", args.lane_vec, args.tile_rows, args.src_tile)
        if args.min_blocks != -1:
            mesh.set_min_blocks(args.min_blocks)
    else:
        mesh.autotune(eps, w.shots, wav, dt, steps=32, level=1)
        # register cap, row sweep, prefetch of the late-loaded rows (and of
        # the next swept block) and the uniformly strided stiffness for the
        # chosen row shape, each timed as the best of three whole runs (the
        # 32-step autotune windows do not always separate them)
        if mesh.tuning()["forward"]["tile_rows"] == 0 and mesh.tuning()["forward"]["tma"] == 0:
            best = None
            for uni in (False, True):
                try:
                    mesh.set_uniform_ell(uni)
                except Exception:           # refused: padding would double K
                    continue
                for cap, sweep, pf in ((0, 0, 0), (0, 4, 0), (5, 0, 0), (5, 4, 0), (5, 4, 2),
                                       (5, 4, 3)):
                    mesh.set_min_blocks(cap)
                    mesh.set_row_sweep(sweep)
                    mesh.set_late_prefetch(pf, "forward")
                    mg.forward(mesh, eps, w.shots, wav, dt)
                    torch.cuda.synchronize()
                    ms = run_ms()
                    if best is None or ms < best[4] * 0.99:
                        best = (uni, cap, sweep, pf, ms)
            uniform = best[0]
            mesh.set_uniform_ell(uniform)
            mesh.set_min_blocks(best[1])
            mesh.set_row_sweep(best[2])
            mesh.set_late_prefetch(best[3], "forward")
    if args is not None and args.dep_launch != -1:
        mesh.set_dependent_launch(args.dep_launch)
    tuning = mesh.tuning()
    tuning["forward"]["uniform"] = int(uniform)
    # chunk-major stiffness entries for the forward's lanes per row
    ch_arg = -1 if args is None else args.chunked_ell
    if args is not None and args.tuning and ch_arg == -1:
        ch_arg = int(json.loads(args.tuning).get("ellc", -1))
    set_chunked(mesh, tuning, 64, ch_arg, "forward")
    mg.forward(mesh, eps, w.shots, wav, dt)            # warm-up (graphs, buffers)
    torch.cuda.synchronize()
    if args is not None and args.profile:
        torch.cuda.profiler.start()
    s = run_ms(1 if args is not None and args.profile else 3) / 1e3
    if args is not None and args.profile:
        torch.cuda.profiler.stop()
    n, S = w.n_nodes, w.shots.n_shots
    info = mesh.info()
    S_pad = 64
    bytes_step = 12.0 * n * S_pad + 8.0 * info["nnz"] + 16.0 * n
    peak, kind = peaks()
    traffic = traffic_for("ellipsoid_3d forward", tuning["forward"], uniform)
    mesh.close()
    return {"workload": f"ellipsoid_3d: {n} nodes, {w.mesh.cells.shape[0]} tets, {S} "
                        f"backscatter shots, {nt} of its 6000 steps timed (forward only; the "
                        f"rate per step does not depend on the step count)",
            "forward_updates_per_s": n * S * nt / s, "us_per_leapfrog_step": 1e6 * s / nt,
            "tuning": tuning["forward"],
            "roofline": roofline(
                "k_step (batched forward leapfrog step)", bytes_step, s / nt, traffic, peak,
                peak_kind_note(kind),
                "bytes in flight: DRAM traffic is the algorithmic bytes (ncu), the kernel is "
                "latency bound (long-scoreboard stalls, issue ~35%)",
                f"best of three runs of {nt} steps, CUDA events on the launching stream")}


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


def pml_leg(mg, torch, mesh, w, eps_d, wav_d, dt, nt=1000, ckpt=1000):
    """The split-field PML path (first-order flux leapfrog with element
    fluxes): forward, J v and J^T w on the bench mesh with the square layer
    of thickness 15% of the half-width (varsigma dt = 1/4), over `nt` steps;
    algorithmic bytes per forward step: p read by the flux update, q read
    and written, q read by the node update, p read and written."""
    stream = torch.cuda.current_stream()
    m = w.mesh
    half = float(np.abs(m.coords).max())
    c = m.coords[m.cells].mean(axis=1)
    a = np.abs(c)
    vs = 0.25 / dt
    xi = np.where(a.max(axis=1) >= 0.85 * half, vs, 0.0)
    zeta = np.where(a >= 0.85 * half, vs, 0.0)
    dev = eps_d.device
    xi_d = torch.as_tensor(xi, dtype=torch.float64, device=dev)
    zeta_d = torch.as_tensor(np.ascontiguousarray(zeta), dtype=torch.float64, device=dev)
    wav = wav_d[:nt].contiguous()
    v = torch.as_tensor(np.random.default_rng(0).standard_normal(m.n_cells[1]),
                        dtype=torch.float64, device=dev)
    calls = {
        "forward": lambda: mg.forward_pml(mesh, eps_d, w.shots, wav, dt, xi_d, zeta_d),
        "tangent": lambda: mg.jacobian_apply_pml(mesh, 1, eps_d, w.shots, wav, dt, v, xi_d,
                                                 zeta_d),
    }
    secs = {}
    y = None
    for name, fn in calls.items():
        out = fn()                                              # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        secs[name] = e0.elapsed_time(e1) / 1e3
        if name == "forward":
            y = out
    fn = lambda: mg.jacobian_T_apply_pml(mesh, 1, eps_d, w.shots, wav, dt, y, xi_d, zeta_d,
                                         ckpt_every=ckpt)
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    secs["adjoint"] = e0.elapsed_time(e1) / 1e3
    n, mc, d = w.n_nodes, len(m.cells), m.coords.shape[1]
    S = w.shots.n_shots
    ld = 4 if S <= 4 else (S + 3) // 4 * 4
    bytes_fwd = 4.0 * ld * (3 * n + 3 * d * mc)
    us = {k: 1e6 * s / nt for k, s in secs.items()}
    return {"workload": f"{w.name} with a square layer (xi, zeta = {vs:.3g} beyond 0.85 of the "
                        f"half-width): {n} nodes, {mc} cells, {S} shots, {nt} steps",
            "seconds": secs, "us_per_step": us,
            "forward_updates_per_s": n * S * nt / secs["forward"],
            "algorithmic_bytes_per_forward_step": bytes_fwd,
            "forward_GB_per_s": bytes_fwd / (us["forward"] * 1e-6) / 1e9,
            "adjoint_vs_forward": secs["adjoint"] / secs["forward"],
            "graphs": mesh.tuning()["chunk"] >= 2,
            "note": f"two launches per step (flux and node updates), whole chunks of "
                    f"{mesh.tuning()['chunk']} steps replayed as CUDA graphs; the adjoint "
                    f"includes its forward, which keeps every state (checkpoint spacing {ckpt} "
                    f">= {nt} steps: one segment, no recompute)"}


def batch_leg(mg, torch, dev, nt=4000, ckpt=256):
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


def tune_kept(mg, torch, mesh, w, eps_d, wav_d, dt, v_d, level, nt_probe=1024):
    """Shot groups and register caps per kind for the kept-history path (the
    states it streams are larger than L2, unlike the checkpointed path the
    autotuner times): the fused forward + tangent pass (keeping the history)
    and J^T w on it are timed over the first nt_probe steps with 1, 2 and 4
    groups under each register cap of the kind's row kernel; the fastest
    stays."""
    stream = torch.cuda.current_stream()
    nt_probe = min(nt_probe, len(wav_d))
    wav = wav_d[:nt_probe].contiguous()
    W = torch.zeros((w.shots.n_traces, nt_probe), dtype=torch.float32, device=eps_d.device)
    calls = {
        # the fused forward + tangent pass (tangent kind) keeps the history
        "tangent": lambda: mg.forward_jacobian_apply(mesh, level, eps_d, w.shots, wav, dt, v_d,
                                                     keep_states=True),
        "adjoint": lambda: mg.jacobian_T_apply(mesh, level, eps_d, w.shots, wav, dt, W,
                                               ckpt_every=nt_probe, reuse_checkpoints=True),
    }
    chosen = {}
    for kind, fn in calls.items():
        best = None
        for cap in {"tangent": (0, 5), "adjoint": (0, 5, 6)}[kind]:
            mesh.set_min_blocks(cap, kind)
            for g in (1, 2, 4):
                mesh.set_shot_groups(g, kind)
                fn()                                   # records the graph
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b)
                if best is None or t < best[1] * 0.99:
                    best = (g, t, cap)
        mesh.set_shot_groups(best[0], kind)
        mesh.set_min_blocks(best[2], kind)
        chosen[kind] = best[0]
        if kind == "tangent":
            calls["tangent"]()                     # kept history for the reverse steps
    mesh.trim()
    return chosen


def guarded(fn, *a, **k):
    """Run one of the auxiliary legs; a failure is reported inside the JSON
    line instead of ending the run."""
    try:
        return fn(*a, **k)
    except Exception as e:                      # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


ORACLE_STEPS = 200      # leapfrog steps of the oracle sample (of the workload's 8000)


def _oracle_shot(task):
    """One worker of the oracle sample: shot `shot` of the bench workload,
    forward + tangent (J e_0) + adjoint (w = its traces) over `nt_s` steps on
    the full mesh, single-threaded.  Returns (seconds, node*shot updates)."""
    shot, nt_s, dt = task
    from oracle import wave

    w = configs.asteroid_2d()
    m = w.mesh
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    sub = w.shots.subset([shot])
    s = w.wavelet(dt, nt_s)
    v = np.zeros(m.n_cells[LEVEL])
    v[0] = 1.0
    de = wave.prolong(v, m.ancestor(LEVEL))
    t0 = time.perf_counter()
    y = wave.forward(pb, dt, s, sub.src, sub.rec_ptr, sub.rec)
    wave.tangent(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, de)
    wave.adjoint_eps(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, y)
    return time.perf_counter() - t0, 3.0 * m.coords.shape[0] * sub.n_shots * nt_s


class OracleSample:
    """The FP64 oracle as it stands, timed on the host's cores: one
    single-threaded process per core (spawned, so that none inherits a CUDA
    context), each running one shot of the bench workload for ORACLE_STEPS
    steps; the rate is the updates of all processes over the slowest one's
    compute time.  A one-process figure is kept beside it."""

    def __init__(self, dt, cores=None):
        import multiprocessing as mp

        self.dt = dt
        self.cores = cores or os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                 "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self):
        tasks = [(k, ORACLE_STEPS, self.dt) for k in range(self.cores)]
        res = self.pool.map(_oracle_shot, tasks, chunksize=1)
        return sum(u for _, u in res) / max(t for t, _ in res), res

    def single(self):
        t, u = self.pool.apply(_oracle_shot, ((0, ORACLE_STEPS, self.dt),))
        return u / t

    def sample_text(self):
        return (f"{self.cores} shots of 128 (one per process, {self.cores} single-threaded "
                f"processes on {self.cores} cores), {ORACLE_STEPS} of 8000 steps each, forward "
                f"+ tangent + adjoint on the full 62,641-node mesh (numpy/scipy FP64)")

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(dt):
    """The oracle's rate on the host's cores (bounded sample, about 10-20 s)."""
    ora = OracleSample(dt)
    try:
        ora.run()                                  # imports and page-in
        val, res = ora.run()
        one = ora.single()
    finally:
        ora.close()
    return {"value": val, "unit": UNIT, "cores": ora.cores, "kind": "oracle",
            "sample": ora.sample_text(), "cores_1_value": one,
            "seconds_per_process": [round(t, 2) for t, _ in res]}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload_for_rank(0, args.nt)
    from oracle import wave

    m = w.mesh
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    dt = w.cfl_fraction * pb.cfl_dt()
    ora = OracleSample(dt)
    try:
        for _ in range(args.warmup):
            ora.run()
        vals = [ora.run()[0] for _ in range(args.steps)]
    finally:
        ora.close()
    # every step is one parallel sample: report its mean rate and time
    val = statistics.mean(vals)
    units = 3.0 * m.coords.shape[0] * ora.cores * ORACLE_STEPS
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * units / val,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": describe(w, "kept")},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": ora.cores, "kind": "oracle",
                         "sample": ora.sample_text()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


def main():
    args = parse()
    relaunch_or_check(args)
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
    if args.dep_launch != -1:
        mesh.set_dependent_launch(args.dep_launch)
    if args.cache_hints != -1:
        mesh.set_cache_hints(args.cache_hints)
    # uniformly strided stiffness copy for the row kernels unless refused
    # (measured +1.7% on this step) or switched off
    uniform = False
    if args.uniform_ell != 0:
        try:
            mesh.set_uniform_ell(True)
            uniform = True
        except mg._lib.MgError:
            if args.uniform_ell == 1:
                raise
    n, S, nt = w.n_nodes, w.shots.n_shots, w.nt
    eps_d = torch.as_tensor(w.eps, dtype=torch.float64, device=dev)
    dt = w.cfl_fraction * mg.cfl_dt(mesh, eps_d)
    wav = w.wavelet(dt)
    wav_d = torch.as_tensor(wav, dtype=torch.float64, device=dev)
    nlev = w.mesh.n_cells[LEVEL]
    v = np.zeros(nlev)
    v[np.random.default_rng(0).integers(nlev)] = 1.0
    v_d = torch.as_tensor(v, dtype=torch.float64, device=dev)
    if args.tuning:
        spec = json.loads(args.tuning)
        apply_tuning(mesh, spec)
        if args.kept_groups == "":    # the groups of the given tuning apply as they are
            args.kept_groups = ",".join(str(spec[k].get("groups", 1))
                                        for k in ("forward", "adjoint", "tangent"))
    elif (args.tile_rows == -1 and args.src_tile == -1 and args.lane_vec == -1
            and not args.no_autotune):
        # launch shapes per kernel kind, timed on this problem (setup, untimed),
        # with the chunk-major entries of the two-float4 row shape in place,
        # so that the shapes that read them are timed as they will run
        if args.chunked_ell != 0:
            s_pad = max(4, 1 << (S - 1).bit_length()) if S <= 128 else (S + 127) // 128 * 128
            c0 = args.chunked_ell if args.chunked_ell > 0 else lanes_per_row(s_pad, 2)
            if 2 <= c0 <= 16 and c0 & (c0 - 1) == 0:
                mesh.set_chunked_ell(c0)
        mesh.autotune(eps_d, w.shots, wav_d, dt, steps=128, level=LEVEL)
    tuning = mesh.tuning()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def allreduce(g):
        if ws > 1:
            pdist.gradient_allreduce(g)
        return g

    # Adjoint strategy of the headline: every forward state kept in HBM when
    # it fits (one segment, no recompute), else checkpoints every CKPT steps.
    S_pad = max(4, 1 << (S - 1).bit_length()) if S <= 128 else (S + 127) // 128 * 128
    states_bytes = 4 * n * S_pad * (nt + 2)
    free_bytes = torch.cuda.mem_get_info(dev)[0]
    keep_states = not args.checkpoints and free_bytes > states_bytes + (16 << 30)
    layout = "kept" if keep_states else "checkpoints"
    kept_groups = None
    if keep_states and args.kept_groups:
        kept_groups = dict(zip(("forward", "adjoint", "tangent"),
                               (int(x) for x in args.kept_groups.split(","))))
        for kind, g in kept_groups.items():
            mesh.set_shot_groups(g, kind)
    elif keep_states and not args.no_autotune:
        kept_groups = tune_kept(mg, torch, mesh, w, eps_d, wav_d, dt, v_d, LEVEL)
    tuning_kept = mesh.tuning()
    # chunk-major stiffness entries for the lanes per row of the kernel that
    # dominates the step (the tangent of the fused pass or of J v)
    chunk = set_chunked(mesh, tuning_kept, S_pad, args.chunked_ell, "tangent")
    mark_chunk(tuning, S_pad, chunk)
    adjoint_mode = (f"every forward state kept in HBM ({states_bytes / 1e9:.1f} GB): J^T w "
                    "without recompute, J v in the forward pass" if keep_states else
                    f"checkpoints every {CKPT} steps, recompute per segment")

    def step_kept():
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        evs[0].record(stream)
        # forward traces and J v in one pass that keeps the history, then
        # J^T w on it (no forward left to run)
        y, _ = mg.forward_jacobian_apply(mesh, LEVEL, eps_d, w.shots, wav_d, dt, v_d,
                                         keep_states=True)
        evs[1].record(stream)
        g = mg.jacobian_T_apply(mesh, LEVEL, eps_d, w.shots, wav_d, dt, y, ckpt_every=nt,
                                reuse_checkpoints=True)
        allreduce(g)
        evs[2].record(stream)
        return evs

    def step_ckpt():
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
        return evs

    def timed_steps(step, K, clocks=False, profile=False):
        """W (>= 3) warm-up steps, then K steps with L2 flushed before each;
        barriers and device synchronisation on both sides."""
        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        clk = clocks_start() if clocks and rank == 0 else None
        l0 = mesh.launch_count()
        if profile:
            torch.cuda.profiler.start()        # profilers capture the timed steps only
        out = []
        for _ in range(K):
            flush.fill_(1.0)                   # evict L2 between timed steps
            out.append(step())
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        if ws > 1:
            torch.distributed.barrier()
        return out, mesh.launch_count() - l0, (clocks_stop(clk, dev.index) if clk else None)

    def total_seconds(times):
        t = sum(e[0].elapsed_time(e[-1]) for e in times) / 1e3
        if ws > 1:
            x = torch.tensor([t], device=dev)
            torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
            t = float(x.item())
        return t

    times, launches, clocks = timed_steps(step_kept if keep_states else step_ckpt, args.steps,
                                          clocks=True, profile=args.profile)
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile": True, "launches": int(launches),
                              "step_ms": [e[0].elapsed_time(e[-1]) for e in times],
                              "tuning": tuning, "kept_groups": kept_groups,
                              "adjoint": adjoint_mode}))
        return 0
    mean_ms = lambda a, b: statistics.mean(e[a].elapsed_time(e[b]) for e in times)
    if keep_states:   # fused forward + tangent pass, then the reverse steps
        phases = {"forward_tangent": mean_ms(0, 1), "adjoint": mean_ms(1, 2)}
    else:
        phases = {"forward": mean_ms(0, 1), "adjoint": mean_ms(1, 2), "tangent": mean_ms(2, 3)}
    total_s = total_seconds(times)
    units_per_step = 3.0 * n * S * nt
    value = units_per_step * args.steps * ws / total_s

    # end to end through the public API with host buffers (pinned), copies inside
    pin = lambda a, dt_: torch.as_tensor(np.ascontiguousarray(a), dtype=dt_).pin_memory().numpy()
    eps_h, wav_h, v_h = pin(w.eps, torch.float64), pin(wav, torch.float64), pin(v, torch.float64)

    def step_host():
        if keep_states:
            y, jv = mg.forward_jacobian_apply(mesh, LEVEL, eps_h, w.shots, wav_h, dt, v_h,
                                              keep_states=True)
        else:
            y = mg.forward(mesh, eps_h, w.shots, wav_h, dt, ckpt_every=CKPT,
                           keep_checkpoints=True)
        g = mg.jacobian_T_apply(mesh, LEVEL, eps_h, w.shots, wav_h, dt, y,
                                ckpt_every=nt if keep_states else CKPT, reuse_checkpoints=True)
        if ws > 1:
            gt = torch.as_tensor(g, device=dev)
            allreduce(gt)
            g = gt.cpu().numpy()
        if not keep_states:
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
    h2d = (2 if keep_states else 3) * (w.eps.nbytes + wav.nbytes) + 4 * R * nt + v.nbytes
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
    # the batched forward alone, for the comparison with one shot at a time
    mg.forward(mesh, eps_d, w.shots, wav_d, dt)
    torch.cuda.synchronize()
    e0.record(stream)
    mg.forward(mesh, eps_d, w.shots, wav_d, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_rate = n * S * nt / (e0.elapsed_time(e1) / 1e3)
    # the kept forward history (up to ~257 GB) is not needed by the legs below
    mesh.trim()
    torch.cuda.empty_cache()

    peak, peak_kind = peaks()
    peak_kind = peak_kind_note(peak_kind)
    info = mesh.info()
    # algorithmic bytes per leapfrog step (all shot groups): states, matrix,
    # per-row coefficients; see the kernel table of the design notes
    b_fwd = 12.0 * n * S_pad + 8.0 * info["nnz"] + 16.0 * n
    b_tan = 24.0 * n * S_pad + 8.0 * info["nnz"] + 24.0 * n
    b_adj = 16.0 * n * S_pad + 8.0 * info["nnz"] + 48.0 * n
    l2_note = ("latency bound with the states L2-resident (ncu: DRAM and L2 at a fifth of their "
               "peaks, long-scoreboard stalls): the fraction is of algorithmic bytes, "
               "dram_frac of the bytes DRAM moved")

    # the same step with C3's memory bound: checkpoints every 256 steps
    c3 = None
    if keep_states and not args.no_c3_leg:
        for kind in ("forward", "tangent", "adjoint"):   # the autotuned groups
            mesh.set_shot_groups(tuning[kind].get("groups", 1), kind)
        tc, _, _ = timed_steps(step_ckpt, max(1, min(args.steps, 2)))
        tcs = total_seconds(tc)
        ph = {"forward": statistics.mean(e[0].elapsed_time(e[1]) for e in tc),
              "adjoint": statistics.mean(e[1].elapsed_time(e[2]) for e in tc),
              "tangent": statistics.mean(e[2].elapsed_time(e[3]) for e in tc)}
        tname = "k_tangent_tiled" if tuning["tangent"]["tile_rows"] else "k_tangent_rows"
        c3 = {"value": units_per_step * len(tc) * ws / tcs, "unit": UNIT,
              "ms_per_step": 1e3 * tcs / len(tc), "phases_ms": ph,
              "workload": describe(w, "checkpoints"), "tuning": tuning,
              "memory": f"checkpoints {2 * ((nt + CKPT - 1) // CKPT) * 4 * n * S_pad / 1e9:.1f} "
                        f"GB + segment {(CKPT + 2) * 4 * n * S_pad / 1e9:.1f} GB",
              "roofline": roofline(
                  f"{tname} (lockstep forward + tangent step, J v)", b_tan,
                  ph["tangent"] / 1e3 / nt,
                  traffic_for("asteroid_2d tangent", tuning["tangent"], uniform), peak,
                  peak_kind, l2_note, "per-step time = J v phase / nt (launch gaps included)",
                  bound=L2_BOUND)}
        mesh.trim()

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
    pml = None if args.no_pml_leg else guarded(pml_leg, mg, torch, mesh, w, eps_d, wav_d, dt)
    mesh.trim()
    batch = None if args.no_batch_leg or ws > 1 else guarded(batch_leg, mg, torch, dev)
    proj["note"] = (f"{R} traces x {nt} samples; FP64 accumulation; inputs L2-resident; "
                    "the projected Jacobian products cost one jacobian_apply / "
                    "jacobian_T_apply each (the forward and adjoint phases above)")

    if rank != 0:
        return 0
    # roofline of the dominant kernel of the headline step: algorithmic bytes
    # per leapfrog step (all shot groups) / (its phase time / nt)
    if keep_states:
        # k_tangent_rows: p_l, p_{l-1}, dp_l, dp_{l-1} read, p_{l+1}, dp_{l+1}
        # written per node.shot; matrix, {alpha, beta, gamma, 1/w} and the
        # tangent coefficients per row
        rf = roofline(
            "k_tangent_rows (fused forward + tangent step, writing the kept history; per "
            "leapfrog step, all shot groups)", b_tan, phases["forward_tangent"] / 1e3 / nt,
            traffic_for("asteroid_2d fused", tuning_kept["tangent"], uniform), peak, peak_kind,
            l2_note, "per-step time = fused phase / nt (includes launch gaps); p_{l+1} is "
                     "written into the kept history in HBM", bound=L2_BOUND)
        adj_rf = roofline(
            "k_adjoint_rows (reverse step on the kept history)", b_adj,
            phases["adjoint"] / 1e3 / nt,
            traffic_for("asteroid_2d reverse", tuning_kept["adjoint"], uniform), peak,
            peak_kind, l2_note, "per-step time = reverse phase / nt", bound=L2_BOUND)
    else:
        rf = roofline("k_step (batched forward leapfrog step)", b_fwd,
                      phases["forward"] / 1e3 / nt,
                      traffic_for("asteroid_2d forward", tuning["forward"], uniform), peak,
                      peak_kind, l2_note, "per-launch time = forward phase / nt",
                      bound=L2_BOUND)
        adj_rf = None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": describe(w, layout), "nodes": n, "shots": S, "nt": nt,
                   "parallelism": f"shots: one 128-shot batch per GPU x {ws}",
                   "tuning": tuning_kept, "adjoint": adjoint_mode, "kept_groups": kept_groups,
                   "stiffness": ("uniformly strided ELL" if uniform else "sliced ELL") + (
                       f", chunk-major copy for {chunk} lanes per row" if chunk else ""),
                   "l2": "flushed between timed steps (256 MB write)"},
        "phases_ms": phases,
        "forward_updates_per_s": fwd_rate,
        "single_source_forward_updates_per_s": single_rate,
        "batched_vs_single_source": fwd_rate / single_rate,
        "roofline": rf,
        "adjoint_roofline": adj_rf,
        "c3_checkpointed": c3,
        "e2e": {"value": units_per_step * e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "projected_data": proj,
        "tv_reconstruction": inversion,
        "approx_jacobian": approx,
        "uneven_batch": batch,
        "pml": pml,
    }
    if not args.no_hbm_leg:
        out["hbm_workload"] = guarded(hbm_leg, mg, torch, dev)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(dt)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
