"""Named synthetic workloads (inputs only).

Each workload fixes the mesh hierarchy, the per-cell permittivity, the shot
geometry, the Ricker centre frequency and the step count.  The time step is
NOT fixed here: it is ``cfl_fraction`` times the CFL bound of the discrete
scheme, which the caller computes with the implementation under test (or
the oracle) and passes back in to ``wavelet``.

  square_disc_2d       [-1,1]^2, 64x64 squares -> 8192 triangles / 4225 nodes,
                       eps=4 with an eps=6 disc, 1 shot x 16 receivers, 2000 steps
  asteroid_2d          asteroid shape, 1944 -> 124,416 triangles (62,641 nodes),
                       layered/elliptic/noisy eps, 128 backscatter shots, 8000 steps
  ellipsoid_3d         ellipsoid 1.0x0.8x0.6, 20,736 -> 10,616,832 tets
                       (1,814,385 nodes), 64 backscatter shots, 6000 steps
  uneven_batch_2d      24 rotated/scaled asteroid instances on levels 1..4 with
                       8..256 shots each, 4000 steps
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import fields, meshes, shots as shots_mod


@dataclasses.dataclass
class Workload:
    name: str
    mesh: meshes.NestedMesh
    eps: np.ndarray           # float64 [n_cells] (finest level)
    shots: shots_mod.Shots
    freq: float               # Ricker centre frequency
    nt: int
    jac_level: int = 1        # mesh level whose cells carry the Jacobian
    cfl_fraction: float = 0.5
    bc: str = "abc"           # "abc" | "neumann" | "dirichlet"

    def wavelet(self, dt: float, nt: int | None = None) -> np.ndarray:
        return shots_mod.ricker(self.freq, dt, self.nt if nt is None else nt)

    @property
    def n_nodes(self) -> int:
        return int(self.mesh.coords.shape[0])


def square_disc_2d(n_coarse=8, n_refine=3, nt=2000, n_rec=16) -> Workload:
    m = meshes.square_mesh(n_coarse, n_refine)
    eps = fields.square_disc_eps(m)
    sh = shots_mod.square_shots(m, n_rec)
    f = shots_mod.ricker_frequency(m.mean_edge_length(), ppw=10.0)
    return Workload("square_disc_2d", m, eps, sh, f, nt)


def asteroid_2d(n_refine=3, K=18, S=128, nt=8000, seed_config=2,
                instance=0, rotation=0.0, scale=1.0, noise=0.05) -> Workload:
    m = meshes.asteroid_mesh(n_refine, K, rotation, scale)
    eps = fields.asteroid_eps(m, seed_config, instance, rotation, scale, noise=noise)
    sh = shots_mod.asteroid_shots(m, S, rotation, scale)
    f = shots_mod.ricker_frequency(m.mean_edge_length(), ppw=10.0)
    return Workload("asteroid_2d", m, eps, sh, f, nt)


def ellipsoid_3d(n_refine=3, grid=meshes.ELLIPSOID_GRID, S=64, nt=6000,
                 seed_config=4) -> Workload:
    m = meshes.ellipsoid_mesh(n_refine, grid)
    eps = fields.ellipsoid_eps(m, seed_config)
    sh = shots_mod.ellipsoid_shots(m, S)
    f = shots_mod.ricker_frequency(m.mean_edge_length(), ppw=8.0)
    return Workload("ellipsoid_3d", m, eps, sh, f, nt)


def uneven_batch_2d(n_instances=24, nt=4000, seed_config=5, K=18,
                    max_level=4) -> list:
    """Instances with level ~ U{1..max_level}, S ~ U{8,...,256}, rotation
    U[0,2pi), scale U[0.75,1.25]; each has its own eps, shots, f and dt."""
    rng = fields.rng_for(seed_config, 999)
    out = []
    for i in range(n_instances):
        lvl = int(rng.integers(1, max_level + 1))
        S = int(rng.choice([8, 16, 32, 64, 128, 256]))
        rot = float(rng.uniform(0.0, 2.0 * math.pi))
        sc = float(rng.uniform(0.75, 1.25))
        w = asteroid_2d(n_refine=lvl, K=K, S=S, nt=nt, seed_config=seed_config,
                        instance=i, rotation=rot, scale=sc)
        w.name = f"uneven_batch_2d[{i}]"
        out.append(w)
    return out


def tiny_2d(n_coarse=2, n_refine=2, nt=120, S=3, seed=7, bc="abc") -> Workload:
    """A few hundred nodes: 2D square with a random eps field, S shots at
    random boundary nodes, each recording at 4 random nodes."""
    m = meshes.square_mesh(n_coarse, n_refine)
    rng = fields.rng_for(0, seed)
    eps = rng.uniform(2.0, 6.0, size=m.cells.shape[0])
    bn = shots_mod.boundary_nodes(m)
    src = rng.choice(bn, size=S, replace=False).astype(np.int32)
    recs = [rng.choice(m.coords.shape[0], size=4, replace=False) for _ in range(S)]
    sh = shots_mod.Shots(src, np.arange(0, 4 * S + 1, 4, dtype=np.int64),
                         np.concatenate(recs).astype(np.int32))
    f = shots_mod.ricker_frequency(m.mean_edge_length(), ppw=10.0)
    return Workload("tiny_2d", m, eps, sh, f, nt, bc=bc)


def tiny_3d(grid=(2, 2, 2), n_refine=1, nt=80, S=3, seed=11, bc="abc") -> Workload:
    m = meshes.ellipsoid_mesh(n_refine, grid)
    rng = fields.rng_for(0, seed)
    eps = rng.uniform(2.0, 6.0, size=m.cells.shape[0])
    bn = shots_mod.boundary_nodes(m)
    src = rng.choice(bn, size=S, replace=False).astype(np.int32)
    recs = [rng.choice(m.coords.shape[0], size=3, replace=False) for _ in range(S)]
    sh = shots_mod.Shots(src, np.arange(0, 3 * S + 1, 3, dtype=np.int64),
                         np.concatenate(recs).astype(np.int32))
    f = shots_mod.ricker_frequency(m.mean_edge_length(), ppw=8.0)
    return Workload("tiny_3d", m, eps, sh, f, nt, bc=bc)


PRESETS = {
    "square_disc_2d": square_disc_2d,
    "asteroid_2d": asteroid_2d,
    "ellipsoid_3d": ellipsoid_3d,
}
