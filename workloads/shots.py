"""Shot geometry (source node + receiver nodes) and the Ricker source wavelet
(inputs only).

A shot places the point source of Eq. (pde1) on a mesh node and records the
potential at a list of receiver nodes.  Prescribed points are snapped to the
nearest boundary node (Euclidean; ties go to the lower node id).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .meshes import ELLIPSOID_AXES, NestedMesh, asteroid_radius


@dataclasses.dataclass
class Shots:
    """src int32 [S]; rec_ptr int64 [S+1]; rec int32 [rec_ptr[-1]]."""

    src: np.ndarray
    rec_ptr: np.ndarray
    rec: np.ndarray

    @property
    def n_shots(self) -> int:
        return int(self.src.shape[0])

    @property
    def n_traces(self) -> int:
        return int(self.rec.shape[0])

    def subset(self, idx) -> "Shots":
        idx = np.asarray(idx, dtype=np.int64)
        recs = [self.rec[self.rec_ptr[i]:self.rec_ptr[i + 1]] for i in idx]
        ptr = np.concatenate([[0], np.cumsum([len(r) for r in recs])]).astype(np.int64)
        rec = np.concatenate(recs).astype(np.int32) if recs else np.zeros(0, np.int32)
        return Shots(self.src[idx].astype(np.int32), ptr, rec)

    def trace_rows(self, idx):
        """Rows of the [n_traces, nt] trace array that belong to shots idx."""
        return np.concatenate([np.arange(self.rec_ptr[i], self.rec_ptr[i + 1])
                               for i in np.asarray(idx)]).astype(np.int64)


def boundary_nodes(mesh: NestedMesh) -> np.ndarray:
    return np.unique(mesh.bnd.ravel()).astype(np.int64)


def nearest_boundary_node(mesh: NestedMesh, points) -> np.ndarray:
    bn = boundary_nodes(mesh)
    pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
    d2 = ((mesh.coords[bn][None, :, :] - pts[:, None, :]) ** 2).sum(-1)
    return bn[np.argmin(d2, axis=1)].astype(np.int32)


def square_shots(mesh: NestedMesh, n_rec: int = 16) -> Shots:
    """One shot: source at the boundary node nearest (-1,0); receivers at the
    boundary nodes nearest the ray/square intersections at angles 2 pi k/n_rec."""
    src = nearest_boundary_node(mesh, [(-1.0, 0.0)])
    th = 2.0 * math.pi * np.arange(n_rec) / n_rec
    d = np.stack([np.cos(th), np.sin(th)], 1)
    pts = d / np.abs(d).max(axis=1, keepdims=True)
    rec = nearest_boundary_node(mesh, pts)
    return Shots(src, np.array([0, n_rec], dtype=np.int64), rec)


def backscatter_shots(src_nodes) -> Shots:
    """Co-located source and receiver per shot (monostatic backscatter)."""
    src = np.asarray(src_nodes, dtype=np.int32)
    return Shots(src, np.arange(src.shape[0] + 1, dtype=np.int64), src.copy())


def asteroid_shots(mesh: NestedMesh, S: int, rotation: float = 0.0,
                   scale: float = 1.0) -> Shots:
    """S backscatter shots at equal angles 2 pi k/S on r(theta)."""
    th = 2.0 * math.pi * np.arange(S) / S
    r = asteroid_radius(th) * scale
    pts = np.stack([r * np.cos(th + rotation), r * np.sin(th + rotation)], 1)
    return backscatter_shots(nearest_boundary_node(mesh, pts))


def ellipsoid_shots(mesh: NestedMesh, S: int, axes=ELLIPSOID_AXES) -> Shots:
    """S backscatter shots on Fibonacci-sphere directions projected onto the
    ellipsoid surface (x = d / |d/axes|)."""
    k = np.arange(S)
    z = 1.0 - (2.0 * k + 1.0) / S
    r = np.sqrt(1.0 - z * z)
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)
    A = np.asarray(axes)
    pts = d / np.sqrt(((d / A[None, :]) ** 2).sum(1))[:, None]
    return backscatter_shots(nearest_boundary_node(mesh, pts))


def ricker_frequency(mean_edge: float, ppw: float, c_bg: float = 0.5) -> float:
    """Centre frequency giving ``ppw`` mean edge lengths per wavelength at
    the background speed c_bg = 1/sqrt(4)."""
    return c_bg / (ppw * mean_edge)


def ricker(f: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Ricker samples s(l dt), l = 0..nt-1, with s(t) = (1 - 2 pi^2 f^2 u^2)
    exp(-pi^2 f^2 u^2), u = t - t0, t0 = 1.5/f by default.  float64."""
    if t0 is None:
        t0 = 1.5 / f
    u = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f * u) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)
