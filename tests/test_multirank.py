"""Two-rank (gloo, CPU) check of the multi-GPU decomposition: shots sharded
round-robin, traces need no exchange, the adjoint gradient is one
all-reduce.  Each rank runs the FP64 oracle on its shard; the result must
equal the unsharded computation."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import wave
from paper_1707_04605_gb300 import distributed as pd
from workloads import configs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = configs.tiny_2d(S=5, nt=80)
        m = w.mesh
        pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
        dt = 0.5 * pb.cfl_dt()
        s = w.wavelet(dt)
        W = np.random.default_rng(9).standard_normal((w.shots.n_traces, len(s)))
        sh, idx = pd.shard(w.shots, rank, world)
        rows = pd.trace_rows(w.shots, idx)
        y = wave.forward(pb, dt, s, sh.src, sh.rec_ptr, sh.rec)
        g = wave.adjoint_eps(pb, dt, s, sh.src, sh.rec_ptr, sh.rec, W[rows])
        gc = wave.restrict(g, m.ancestor(1), m.n_cells[1])
        gt = pd.gradient_allreduce(torch.from_numpy(gc))
        np.save(os.path.join(out_dir, f"y{rank}.npy"), y)
        np.save(os.path.join(out_dir, f"rows{rank}.npy"), rows)
        if rank == 0:
            np.save(os.path.join(out_dir, "g.npy"), gt.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_shot_sharding(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    w = configs.tiny_2d(S=5, nt=80)
    m = w.mesh
    pb = wave.Problem(m.coords, m.cells, m.bnd, w.eps, w.bc)
    dt = 0.5 * pb.cfl_dt()
    s = w.wavelet(dt)
    W = np.random.default_rng(9).standard_normal((w.shots.n_traces, len(s)))
    y = wave.forward(pb, dt, s, w.shots.src, w.shots.rec_ptr, w.shots.rec)
    g = wave.restrict(wave.adjoint_eps(pb, dt, s, w.shots.src, w.shots.rec_ptr, w.shots.rec, W),
                      m.ancestor(1), m.n_cells[1])
    seen = np.zeros(len(y), bool)
    for r in range(world):
        rows = np.load(tmp_path / f"rows{r}.npy")
        assert np.array_equal(np.load(tmp_path / f"y{r}.npy"), y[rows])
        seen[rows] = True
    assert seen.all()
    gr = np.load(tmp_path / "g.npy")
    assert np.abs(gr - g).max() <= 1e-12 * np.abs(g).max()


def test_shard_partition_is_exact():
    w = configs.asteroid_2d(n_refine=1, S=13, nt=10)
    for world in (1, 2, 3, 4):
        rows_all = []
        for r in range(world):
            sh, idx = pd.shard(w.shots, r, world)
            rows = pd.trace_rows(w.shots, idx)
            assert sh.n_shots == len(idx) and sh.n_traces == len(rows)
            assert np.array_equal(sh.src, w.shots.src[idx])
            rows_all.append(rows)
        assert np.array_equal(np.sort(np.concatenate(rows_all)), np.arange(w.shots.n_traces))
