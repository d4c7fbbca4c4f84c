"""Write the stored oracle values of the full-length parity tests.

Every number written here comes from the FP64 oracle (``oracle/wave.py``)
run on the seeded workloads of ``workloads/``; nothing is read from the CUDA
library.  The GPU tests (``tests/test_gpu_full_length.py``) compare the
CUDA path with these files, and ``tests/test_golden.py`` checks, without a
GPU, that the stored oracle tangent agrees with the stored oracle central
differences.

Files (float32 payloads, float64 scalars; each carries fingerprints of its
inputs so a test can tell a changed workload generator from a wrong kernel):

  c4_ellipsoid_3d_traces.npz   ellipsoid_3d (1,814,385 nodes, 10.6M tets):
      the traces of shots 0 and 40 over all 6000 steps (App. A, Eqs.
      (leap-frog1)-(leap-frog2) with the flux eliminated).
  c3_asteroid_2d_jacobian.npz  asteroid_2d (62,641 nodes, 8000 steps),
      shots 0 and 64: 20 seeded level-1 columns J e_j (the auxiliary system
      of App. A.1, Eqs. (aku_ankka), (linearized1)-(linearized2)); the same
      columns by central differences of the forward with h = 1e-3; and one
      level-1 gradient J^T w for seeded weights w on those two traces.
  c5_uneven_batch_2d.npz       the 24 instances of uneven_batch_2d (4000
      steps): per instance one seeded shot's trace and the level-1 gradient
      of seeded weights on that trace alone.

Usage:  python tests/golden/make_golden.py [--only c3,c4,c5] [--procs N]
(about 20 minutes on 8 cores; peak memory about 40 GB).
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

C3_SHOTS = [0, 64]
C3_LEVEL = 1
C3_N_COLS = 20
C3_H = 1e-3
C3_CELL_SEED = 3020
C3_W_SEED = 3021
C4_SHOTS = [0, 40]
C5_LEVEL = 1
C5_SEED = 5000


def fingerprint(w) -> dict:
    """Sums of the inputs both sides read (coordinates, permittivity, shot
    nodes) and the Ricker frequency."""
    m = w.mesh
    return {"fp_n_nodes": np.int64(m.coords.shape[0]),
            "fp_n_cells": np.int64(m.cells.shape[0]),
            "fp_coords_sum": np.float64(np.abs(m.coords).sum()),
            "fp_eps_sum": np.float64(w.eps.sum()),
            "fp_eps_sq_sum": np.float64((w.eps * w.eps).sum()),
            "fp_src": w.shots.src.astype(np.int64),
            "fp_rec": w.shots.rec.astype(np.int64),
            "fp_freq": np.float64(w.freq)}


def _problem(w, eps=None):
    from oracle import wave

    m = w.mesh
    return wave.Problem(m.coords, m.cells, m.bnd, w.eps if eps is None else eps, w.bc)


# ----------------------------------------------------------------- tasks
def task_c4():
    from oracle import wave
    from workloads import configs

    w = configs.ellipsoid_3d()
    pb = _problem(w)
    dt = w.cfl_fraction * pb.cfl_dt()
    s = w.wavelet(dt)
    sub = w.shots.subset(C4_SHOTS)
    y = wave.forward(pb, dt, s, sub.src, sub.rec_ptr, sub.rec)
    return "c4", None, {"dt": dt, "traces": y, **fingerprint(w)}


def _c3_setup():
    from workloads import configs

    w = configs.asteroid_2d()
    pb = _problem(w)
    dt = w.cfl_fraction * pb.cfl_dt()
    nl = w.mesh.n_cells[C3_LEVEL]
    cells = np.random.default_rng(C3_CELL_SEED).choice(nl, size=C3_N_COLS, replace=False)
    return w, pb, dt, cells


def task_c3_tangent(j):
    from oracle import wave

    w, pb, dt, cells = _c3_setup()
    sub = w.shots.subset(C3_SHOTS)
    v = np.zeros(w.mesh.n_cells[C3_LEVEL])
    v[cells[j]] = 1.0
    de = wave.prolong(v, w.mesh.ancestor(C3_LEVEL))
    dy = wave.tangent(pb, dt, w.wavelet(dt), sub.src, sub.rec_ptr, sub.rec, de)
    return "c3_tan", j, dy


def task_c3_fd(j):
    """Central difference (y(eps + h e_j) - y(eps - h e_j)) / 2h of the
    oracle forward, e_j the prolonged indicator of level cell j."""
    from oracle import wave

    w, pb, dt, cells = _c3_setup()
    sub = w.shots.subset(C3_SHOTS)
    v = np.zeros(w.mesh.n_cells[C3_LEVEL])
    v[cells[j]] = 1.0
    de = wave.prolong(v, w.mesh.ancestor(C3_LEVEL))
    s = w.wavelet(dt)
    ys = []
    for sign in (1.0, -1.0):
        pbh = _problem(w, w.eps + sign * C3_H * de)
        ys.append(wave.forward(pbh, dt, s, sub.src, sub.rec_ptr, sub.rec))
    return "c3_fd", j, (ys[0] - ys[1]) / (2.0 * C3_H)


def task_c3_gradient():
    from oracle import wave

    w, pb, dt, cells = _c3_setup()
    sub = w.shots.subset(C3_SHOTS)
    W = np.random.default_rng(C3_W_SEED).standard_normal((sub.n_traces, w.nt)).astype(np.float32)
    s = w.wavelet(dt)
    y = wave.forward(pb, dt, s, sub.src, sub.rec_ptr, sub.rec)
    g = wave.adjoint_eps(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, W.astype(np.float64))
    gl = wave.restrict(g, w.mesh.ancestor(C3_LEVEL), w.mesh.n_cells[C3_LEVEL])
    return "c3_grad", None, {"dt": dt, "cells": cells.astype(np.int64), "weights": W,
                             "gradient": gl, "traces": y, **fingerprint(w)}


def c5_pick(i, n_shots, nt):
    """The sampled shot of instance i and its seeded trace weights."""
    rng = np.random.default_rng(C5_SEED + i)
    shot = int(rng.integers(n_shots))
    return shot, rng.standard_normal(nt).astype(np.float32)


def task_c5(i):
    from oracle import wave
    from workloads import configs

    w = configs.uneven_batch_2d()[i]
    pb = _problem(w)
    dt = w.cfl_fraction * pb.cfl_dt()
    s = w.wavelet(dt)
    shot, Wv = c5_pick(i, w.shots.n_shots, w.nt)
    sub = w.shots.subset([shot])
    y = wave.forward(pb, dt, s, sub.src, sub.rec_ptr, sub.rec)
    W = np.repeat(Wv[None, :].astype(np.float64), sub.n_traces, axis=0)
    g = wave.adjoint_eps(pb, dt, s, sub.src, sub.rec_ptr, sub.rec, W)
    gl = wave.restrict(g, w.mesh.ancestor(C5_LEVEL), w.mesh.n_cells[C5_LEVEL])
    fp = fingerprint(w)
    return "c5", i, {"dt": dt, "shot": shot, "weights": Wv, "traces": y, "gradient": gl,
                     "fp_eps_sum": fp["fp_eps_sum"], "fp_coords_sum": fp["fp_coords_sum"],
                     "fp_n_nodes": fp["fp_n_nodes"]}


def _run(task):
    fn, args = task
    t0 = time.time()
    out = fn(*args)
    print(f"  {fn.__name__}{args} done in {time.time() - t0:.0f} s", flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="c3,c4,c5")
    ap.add_argument("--procs", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    want = set(args.only.split(","))
    tasks = []
    if "c4" in want:
        tasks.append((task_c4, ()))
    if "c3" in want:
        tasks.append((task_c3_gradient, ()))
        tasks += [(task_c3_tangent, (j,)) for j in range(C3_N_COLS)]
        tasks += [(task_c3_fd, (j,)) for j in range(C3_N_COLS)]
    if "c5" in want:
        tasks += [(task_c5, (i,)) for i in range(24)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs, maxtasksperchild=1) as pool:
        results = pool.map(_run, tasks, chunksize=1)
    tan, fd, c5 = {}, {}, {}
    c3 = None
    for kind, j, val in results:
        if kind == "c4":
            np.savez_compressed(os.path.join(HERE, "c4_ellipsoid_3d_traces.npz"),
                                shots=np.array(C4_SHOTS), **{**val, "traces":
                                                               val["traces"].astype(np.float32)})
        elif kind == "c3_tan":
            tan[j] = val
        elif kind == "c3_fd":
            fd[j] = val
        elif kind == "c3_grad":
            c3 = val
        elif kind == "c5":
            c5[j] = val
    if c3 is not None:
        cols = np.stack([tan[j] for j in range(C3_N_COLS)]).astype(np.float32)
        fds = np.stack([fd[j] for j in range(C3_N_COLS)]).astype(np.float32)
        np.savez_compressed(os.path.join(HERE, "c3_asteroid_2d_jacobian.npz"),
                            shots=np.array(C3_SHOTS), level=np.int64(C3_LEVEL),
                            h=np.float64(C3_H), columns=cols, fd_columns=fds,
                            **{**c3, "traces": c3["traces"].astype(np.float32)})
    if c5:
        n = len(c5)
        np.savez_compressed(
            os.path.join(HERE, "c5_uneven_batch_2d.npz"),
            level=np.int64(C5_LEVEL),
            dt=np.array([c5[i]["dt"] for i in range(n)]),
            shot=np.array([c5[i]["shot"] for i in range(n)], dtype=np.int64),
            weights=np.stack([c5[i]["weights"] for i in range(n)]),
            traces=np.stack([c5[i]["traces"][0] for i in range(n)]).astype(np.float32),
            gradient=np.concatenate([c5[i]["gradient"] for i in range(n)]).astype(np.float32),
            gradient_ptr=np.cumsum([0] + [len(c5[i]["gradient"]) for i in range(n)]),
            fp_eps_sum=np.array([c5[i]["fp_eps_sum"] for i in range(n)]),
            fp_coords_sum=np.array([c5[i]["fp_coords_sum"] for i in range(n)]),
            fp_n_nodes=np.array([c5[i]["fp_n_nodes"] for i in range(n)]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
