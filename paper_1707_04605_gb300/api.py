"""Python binding of the C ABI (argument marshalling only).

Every function mirrors one entry point of include/mgwave.h.  Array
arguments are either all CUDA tensors (device mode: work is queued on the
current torch stream, results are CUDA tensors) or all host arrays (host
mode, MG_HOST_PTRS: the library copies in and out itself and returns host
arrays).  Nothing here computes any part of the wave path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _is_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _stream_ptr(stream):
    if stream is not None:
        return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch

    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _host(x, dtype):
    a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
    return a, C.c_void_p(a.ctypes.data)


def _dev(x, dtype_name):
    import torch

    want = {"float64": torch.float64, "float32": torch.float32}[dtype_name]
    if x.dtype != want:
        raise TypeError(f"expected a {dtype_name} CUDA tensor, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError("CUDA tensor arguments must be contiguous")
    return x, C.c_void_p(x.data_ptr())


class Shots:
    """Host-side shot batch (mg_shots): src [S] int32, rec_ptr [S+1] int64,
    rec [R] int32 in caller node ids."""

    def __init__(self, src, rec_ptr, rec):
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.rec_ptr = np.ascontiguousarray(rec_ptr, dtype=np.int64)
        self.rec = np.ascontiguousarray(rec, dtype=np.int32)
        self.c = L.mg_shots(
            len(self.src),
            self.src.ctypes.data_as(C.POINTER(C.c_int32)),
            self.rec_ptr.ctypes.data_as(C.POINTER(C.c_int64)),
            self.rec.ctypes.data_as(C.POINTER(C.c_int32)))

    @property
    def n_shots(self) -> int:
        return int(self.src.shape[0])

    @property
    def n_traces(self) -> int:
        return int(self.rec_ptr[-1])

    @classmethod
    def of(cls, shots) -> "Shots":
        if isinstance(shots, Shots):
            return shots
        return cls(shots.src, shots.rec_ptr, shots.rec)


class Mesh:
    """Handle of mg_mesh_create; destroyed with the object or by close()."""

    def __init__(self, handle, dim, n_cells_per_level):
        self._h = handle
        self.dim = dim
        self.n_cells_per_level = [int(x) for x in n_cells_per_level]
        self._lib = L.load()

    @property
    def handle(self):
        if not self._h:
            raise ValueError("mesh handle is closed")
        return self._h

    def close(self):
        if self._h:
            self._lib.mg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = L.mg_mesh_info_t()
        L.check(self._lib.mg_mesh_get_info(self.handle, C.byref(inf)), "mg_mesh_get_info")
        return {k: getattr(inf, k) for k, _ in L.mg_mesh_info_t._fields_}

    def permutation(self) -> np.ndarray:
        n = self.info()["n_nodes"]
        out = np.empty(n, dtype=np.int32)
        L.check(self._lib.mg_mesh_get_permutation(self.handle, C.c_void_p(out.ctypes.data)),
                "mg_mesh_get_permutation")
        return out

    def trim(self):
        L.check(self._lib.mg_mesh_trim(self.handle), "mg_mesh_trim")

    def checkpoint_generation(self) -> int:
        """mg_mesh_checkpoint_generation: changes whenever the handle's
        checkpoints or kept states are written or dropped."""
        return int(self._lib.mg_mesh_checkpoint_generation(self.handle))

    def launch_count(self) -> int:
        return int(self._lib.mg_launch_count(self.handle))

    KINDS = {"forward": 0, "tangent": 1, "adjoint": 2}

    def set_kernel_tuning(self, kind: str, batch: int = -1, tile_rows: int = -1,
                          src_tile: int = -1):
        L.check(self._lib.mg_mesh_set_kernel_tuning(self.handle, self.KINDS[kind], int(batch),
                                                    int(tile_rows), int(src_tile)),
                "mg_mesh_set_kernel_tuning")

    def set_shot_groups(self, groups: int, kind: str = None):
        """Shot groups advanced one after another per graph chunk / checkpoint
        segment (mg_mesh_set_shot_groups); kind None sets all kinds."""
        k = -1 if kind is None else self.KINDS[kind]
        L.check(self._lib.mg_mesh_set_shot_groups(self.handle, k, int(groups)),
                "mg_mesh_set_shot_groups")

    def set_conductivity(self, sigma, stream=None):
        """Per-cell conductivity (mg_mesh_set_conductivity); None removes it."""
        if sigma is None:
            rc = self._lib.mg_mesh_set_conductivity(self.handle, None, None, 0)
        elif _is_cuda(sigma):
            sigma, ps = _dev(sigma, "float64")
            rc = self._lib.mg_mesh_set_conductivity(self.handle, ps, _stream_ptr(stream), 0)
        else:
            sigma, ps = _host(sigma, np.float64)
            rc = self._lib.mg_mesh_set_conductivity(self.handle, ps, None, L.MG_HOST_PTRS)
        L.check(rc, "mg_mesh_set_conductivity")

    def set_gather_ring(self, depth: int, kind=None):
        """Gather ring of the row kernels (mg_mesh_set_gather_ring): depth 0,
        4 or 8 for one kind ("forward", "tangent", "adjoint") or all (None)."""
        k = -1 if kind is None else self.KINDS[kind]
        L.check(self._lib.mg_mesh_set_gather_ring(self.handle, int(k), int(depth)),
                "mg_mesh_set_gather_ring")

    def set_l1_streaming(self, on: bool, kind=None):
        """Once-read loads of the row kernels without L1 allocation
        (mg_mesh_set_l1_streaming) for one kind or all (None)."""
        k = -1 if kind is None else self.KINDS[kind]
        L.check(self._lib.mg_mesh_set_l1_streaming(self.handle, int(k), int(bool(on))),
                "mg_mesh_set_l1_streaming")

    def set_tma_tiles(self, rows: int):
        """Rows per tile of the bulk-copy tiled forward (mg_mesh_set_tma_tiles);
        0: off."""
        L.check(self._lib.mg_mesh_set_tma_tiles(self.handle, int(rows)),
                "mg_mesh_set_tma_tiles")

    def set_late_prefetch(self, level: int, kind: str = None):
        """Prefetch (0 none, 1 L1, 2 L2) of the rows the register-capped row
        kernels load after their gathers (mg_mesh_set_late_prefetch); kind
        None sets all kinds."""
        k = -1 if kind is None else self.KINDS[kind]
        L.check(self._lib.mg_mesh_set_late_prefetch(self.handle, k, int(level)),
                "mg_mesh_set_late_prefetch")

    def set_wide_lanes(self, on: bool):
        """8 consecutive shots per lane (32-byte gathers) in the capped
        forward row kernel with two float4 per lane (mg_mesh_set_wide_lanes)."""
        L.check(self._lib.mg_mesh_set_wide_lanes(self.handle, int(bool(on))),
                "mg_mesh_set_wide_lanes")

    def set_chunked_ell(self, chunk: int):
        """Chunk-major copy of the stiffness entries for the wide-lane forward
        with `chunk` lanes per row (mg_mesh_set_chunked_ell); 0: off."""
        L.check(self._lib.mg_mesh_set_chunked_ell(self.handle, int(chunk)),
                "mg_mesh_set_chunked_ell")

    def set_row_sweep(self, blocks: int):
        """Consecutive row blocks per CTA of the forward row kernel
        (mg_mesh_set_row_sweep); 0 or 1: one."""
        L.check(self._lib.mg_mesh_set_row_sweep(self.handle, int(blocks)),
                "mg_mesh_set_row_sweep")

    def set_persistent(self, steps: int = 128, wait_cycles: int = 1 << 31,
                       extra_arrivals: int = 0):
        """Steps per cooperative launch of the MG_PERSISTENT forward, the SM
        clock cycles one grid-barrier wait may take, and (tests only) barrier
        arrivals awaited beyond the grid (mg_mesh_set_persistent)."""
        L.check(self._lib.mg_mesh_set_persistent(self.handle, int(steps), int(wait_cycles),
                                                 int(extra_arrivals)), "mg_mesh_set_persistent")

    def set_min_blocks(self, min_blocks: int, kind: str = "forward"):
        """Register cap of the forward, tangent or adjoint row kernel
        (mg_mesh_set_min_blocks / mg_mesh_set_kernel_min_blocks): 0 or 5,
        or 6 for the adjoint."""
        if kind != "forward":
            L.check(self._lib.mg_mesh_set_kernel_min_blocks(self.handle, self.KINDS[kind],
                                                            int(min_blocks)),
                    "mg_mesh_set_kernel_min_blocks")
            return
        L.check(self._lib.mg_mesh_set_min_blocks(self.handle, int(min_blocks)),
                "mg_mesh_set_min_blocks")

    def set_bulk_copies(self, on: bool):
        """Forward step with bulk-copied neighbour rows (mg_mesh_set_bulk_copies)."""
        L.check(self._lib.mg_mesh_set_bulk_copies(self.handle, int(bool(on))),
                "mg_mesh_set_bulk_copies")

    def set_uniform_ell(self, on: bool):
        """Uniformly strided stiffness copy for the row kernels
        (mg_mesh_set_uniform_ell); same results."""
        L.check(self._lib.mg_mesh_set_uniform_ell(self.handle, int(bool(on))),
                "mg_mesh_set_uniform_ell")

    def set_cache_hints(self, on: bool):
        """L2 evict-first on the last reads of kept states
        (mg_mesh_set_cache_hints); results unchanged."""
        L.check(self._lib.mg_mesh_set_cache_hints(self.handle, int(bool(on))),
                "mg_mesh_set_cache_hints")

    def set_dependent_launch(self, on: bool):
        """Row kernels launched as programmatic dependents of the previous
        kernel (mg_mesh_set_dependent_launch); bit-identical results."""
        L.check(self._lib.mg_mesh_set_dependent_launch(self.handle, int(bool(on))),
                "mg_mesh_set_dependent_launch")

    def device_status(self) -> int:
        """mg_mesh_device_status: 0, or the MG_ERR_* code of a failed bounded wait."""
        return int(self._lib.mg_mesh_device_status(self.handle))

    def tuning(self) -> dict:
        out = np.zeros(17, dtype=np.int32)
        L.check(self._lib.mg_mesh_get_tuning(self.handle, C.c_void_p(out.ctypes.data)),
                "mg_mesh_get_tuning")
        d = {"chunk": int(out[0])}
        for name, k in self.KINDS.items():
            d[name] = {"batch": int(out[1 + 5 * k]), "tile_rows": int(out[2 + 5 * k]),
                       "src_tile": int(out[3 + 5 * k]), "groups": int(out[4 + 5 * k]),
                       "min_blocks": int(out[5 + 5 * k])}
        d["forward"]["bulk"] = int(out[16])
        ring = np.zeros(3, dtype=np.int32)
        L.check(self._lib.mg_mesh_get_gather_ring(self.handle, C.c_void_p(ring.ctypes.data)),
                "mg_mesh_get_gather_ring")
        for name, k in self.KINDS.items():
            d[name]["ring"] = int(ring[k])
        d["forward"]["sweep"] = int(self._lib.mg_mesh_get_row_sweep(self.handle))
        d["forward"]["wide"] = int(self._lib.mg_mesh_get_wide_lanes(self.handle))
        pf = (C.c_int32 * 3)()
        L.check(self._lib.mg_mesh_get_late_prefetch(self.handle, pf), "mg_mesh_get_late_prefetch")
        for k, kind in enumerate(("forward", "tangent", "adjoint")):
            d[kind]["prefetch"] = int(pf[k])
        d["forward"]["tma"] = int(self._lib.mg_mesh_get_tma_tiles(self.handle))
        l1 = np.zeros(3, dtype=np.int32)
        L.check(self._lib.mg_mesh_get_l1_streaming(self.handle, C.c_void_p(l1.ctypes.data)),
                "mg_mesh_get_l1_streaming")
        for name, k in self.KINDS.items():
            d[name]["stream"] = int(l1[k])
        return d

    def autotune(self, eps, shots, wavelet, dt, steps=128, level=1, allow_cfl=False,
                 stream=None) -> dict:
        """Time the candidate launch shapes per kernel kind (mg_autotune) on
        CUDA inputs and keep the fastest; returns the chosen tuning."""
        sh = Shots.of(shots)
        eps, pe = _dev(eps, "float64")
        wavelet, pw = _dev(wavelet, "float64")
        out = np.zeros(17, dtype=np.int32)
        L.check(self._lib.mg_autotune(self.handle, pe, C.byref(sh.c), pw, float(dt), int(steps),
                                      int(level), _stream_ptr(stream),
                                      L.MG_ALLOW_CFL if allow_cfl else 0,
                                      C.c_void_p(out.ctypes.data)), "mg_autotune")
        return self.tuning()

    def set_tuning(self, chunk: int = -1, batch: int = -1, tile_rows: int = -1,
                   src_tile: int = -1):
        """Graph chunk length (even, 0 = plain launches), untiled gather batch
        (4/8), shared-memory tile rows (multiple of 32, 0 = untiled) and shots
        per staged pass (4..64); -1 keeps a value."""
        L.check(self._lib.mg_mesh_set_tuning(self.handle, int(chunk), int(batch),
                                             int(tile_rows), int(src_tile)),
                "mg_mesh_set_tuning")


def mesh_create(dim, coords, cells, cell_parent, n_cells_per_level, bnd, bc="abc",
                order="morton") -> Mesh:
    lib = L.load()
    coords, pc = _host(coords, np.float64)
    cells, pcells = _host(cells, np.int32)
    bnd, pb = _host(bnd, np.int32)
    ncl, pncl = _host(n_cells_per_level, np.int64)
    parents = [np.ascontiguousarray(p, dtype=np.int32) for p in (cell_parent or [])]
    arr = (C.c_void_p * max(1, len(parents)))(*[p.ctypes.data for p in parents])
    h = C.c_void_p()
    rc = lib.mg_mesh_create(int(dim), len(ncl), pc, coords.shape[0], pcells, cells.shape[0],
                            C.cast(arr, C.c_void_p) if parents else None, pncl, pb,
                            bnd.shape[0], L.MG_BC[bc], L.MG_ORDER[order], C.byref(h))
    L.check(rc, "mg_mesh_create")
    return Mesh(h, dim, ncl)


def mesh_from_workload(w, order="morton", bc=None) -> Mesh:
    m = w.mesh
    return mesh_create(m.dim, m.coords, m.cells, m.cell_parent, m.n_cells, m.bnd,
                       bc or w.bc, order)


def cfl_dt(mesh: Mesh, eps, stream=None) -> float:
    lib = L.load()
    out = C.c_double()
    if _is_cuda(eps):
        eps, pe = _dev(eps, "float64")
        rc = lib.mg_cfl_dt(mesh.handle, pe, 0, _stream_ptr(stream), C.byref(out))
    else:
        eps, pe = _host(eps, np.float64)
        rc = lib.mg_cfl_dt(mesh.handle, pe, L.MG_HOST_PTRS, None, C.byref(out))
    L.check(rc, "mg_cfl_dt")
    return float(out.value)


def _prep(eps, wavelet, extra, stream):
    """Marshal eps (float64), wavelet (float64) and extra arrays."""
    if _is_cuda(eps):
        eps, pe = _dev(eps, "float64")
        wavelet, pw = _dev(wavelet, "float64")
        ex = [_dev(x, dt) for x, dt in extra]
        return True, (eps, pe), (wavelet, pw), ex, _stream_ptr(stream), 0
    eps, pe = _host(eps, np.float64)
    wavelet, pw = _host(wavelet, np.float64)
    ex = [_host(x, np.dtype(dt)) for x, dt in extra]
    return False, (eps, pe), (wavelet, pw), ex, None, L.MG_HOST_PTRS


def _alloc(device, shape, dtype_name, like):
    if device:
        import torch

        return torch.empty(shape, dtype=getattr(torch, dtype_name), device=like.device)
    return np.empty(shape, dtype=np.dtype(dtype_name))


def _ptr(x):
    return C.c_void_p(x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data)


def forward(mesh: Mesh, eps, shots, wavelet, dt, nt=None, *, ckpt_every=0,
            keep_checkpoints=False, keep_states=False, single_source=False, allow_cfl=False,
            persistent=False, stream=None, flags=0):
    """Traces [n_traces, nt] float32 of mg_forward.  keep_states keeps every
    state in the handle (MG_KEEP_STATES; (nt + 2) n S_pad floats), so that
    jacobian_T_apply(..., ckpt_every=nt, reuse_checkpoints=True) runs no
    recompute.  persistent runs several steps per cooperative launch
    (MG_PERSISTENT; see Mesh.set_persistent)."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    dev, (eps, pe), (wav, pw), _, st, f0 = _prep(eps, wavelet, [], stream)
    out = _alloc(dev, (sh.n_traces, nt), "float32", eps)
    f = f0 | flags
    if keep_checkpoints:
        f |= L.MG_KEEP_CHECKPOINTS
    if keep_states:
        f |= L.MG_KEEP_STATES
    if single_source:
        f |= L.MG_SINGLE_SOURCE
    if allow_cfl:
        f |= L.MG_ALLOW_CFL
    if persistent:
        f |= L.MG_PERSISTENT
    rc = lib.mg_forward(mesh.handle, pe, C.byref(sh.c), pw, float(dt), nt, _ptr(out),
                        int(ckpt_every), st, f)
    L.check(rc, "mg_forward")
    return out


def jacobian_apply(mesh: Mesh, level, eps, shots, wavelet, dt, v, nt=None, *,
                   reuse_states=False, allow_cfl=False, stream=None, flags=0):
    """J v: tangent traces [n_traces, nt] float32 for a level-cell direction v.
    reuse_states reads the forward field kept by forward(..., keep_states=True)
    (same inputs) instead of recomputing it."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    dev, (eps, pe), (wav, pw), ex, st, f0 = _prep(eps, wavelet, [(v, "float64")], stream)
    (v, pv), = ex
    out = _alloc(dev, (sh.n_traces, nt), "float32", eps)
    f = f0 | flags | (L.MG_ALLOW_CFL if allow_cfl else 0)
    if reuse_states:
        f |= L.MG_REUSE_CHECKPOINTS
    rc = lib.mg_jacobian_apply(mesh.handle, int(level), pe, C.byref(sh.c), pw, float(dt), nt,
                               pv, _ptr(out), st, f)
    L.check(rc, "mg_jacobian_apply")
    return out


def forward_jacobian_apply(mesh: Mesh, level, eps, shots, wavelet, dt, v, nt=None, *,
                           keep_states=False, allow_cfl=False, persistent=False, stream=None,
                           flags=0):
    """(traces, J v) of one fused pass (mg_forward_jacobian_apply); with
    keep_states the forward history stays in the handle for
    jacobian_T_apply(..., ckpt_every=nt, reuse_checkpoints=True).
    persistent (with keep_states) runs several steps per cooperative launch."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    dev, (eps, pe), (wav, pw), ex, st, f0 = _prep(eps, wavelet, [(v, "float64")], stream)
    (v, pv), = ex
    y = _alloc(dev, (sh.n_traces, nt), "float32", eps)
    jv = _alloc(dev, (sh.n_traces, nt), "float32", eps)
    f = f0 | flags | (L.MG_ALLOW_CFL if allow_cfl else 0)
    if keep_states:
        f |= L.MG_KEEP_STATES
    if persistent:
        f |= L.MG_PERSISTENT
    rc = lib.mg_forward_jacobian_apply(mesh.handle, int(level), pe, C.byref(sh.c), pw,
                                       float(dt), nt, pv, _ptr(y), _ptr(jv), st, f)
    L.check(rc, "mg_forward_jacobian_apply")
    return y, jv


def jacobian_T_apply(mesh: Mesh, level, eps, shots, wavelet, dt, w, nt=None, *,
                     ckpt_every=256, reuse_checkpoints=False, allow_cfl=False,
                     persistent=False, stream=None, flags=0):
    """J^T w: gradient [cells of level] float64 for trace weights w [n_traces, nt]."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    dev, (eps, pe), (wav, pw), ex, st, f0 = _prep(eps, wavelet, [(w, "float32")], stream)
    (w, pwt), = ex
    out = _alloc(dev, (mesh.n_cells_per_level[level],), "float64", eps)
    f = f0 | flags | (L.MG_ALLOW_CFL if allow_cfl else 0)
    if persistent:
        f |= L.MG_PERSISTENT
    if reuse_checkpoints:
        f |= L.MG_REUSE_CHECKPOINTS
    rc = lib.mg_jacobian_T_apply(mesh.handle, int(level), pe, C.byref(sh.c), pw, float(dt),
                                 nt, pwt, _ptr(out), int(ckpt_every), st, f)
    L.check(rc, "mg_jacobian_T_apply")
    return out


def prolong(mesh: Mesh, level, v, base=None, stream=None):
    """Finest-cell values base[e] + v[anc_level(e)] (mg_prolong)."""
    lib = L.load()
    m = mesh.n_cells_per_level[-1]
    if _is_cuda(v):
        v, pv = _dev(v, "float64")
        pb = _dev(base, "float64")[1] if base is not None else None
        out = _alloc(True, (m,), "float64", v)
        rc = lib.mg_prolong(mesh.handle, int(level), pv, pb, _ptr(out), _stream_ptr(stream), 0)
    else:
        v, pv = _host(v, np.float64)
        bh = _host(base, np.float64) if base is not None else (None, None)
        out = np.empty(m, dtype=np.float64)
        rc = lib.mg_prolong(mesh.handle, int(level), pv, bh[1], _ptr(out), None, L.MG_HOST_PTRS)
    L.check(rc, "mg_prolong")
    return out


def _traces_pair(a, b, b_dtype):
    """Marshal a [R, nt] float32 and a second array of dtype b_dtype."""
    if _is_cuda(a):
        a, pa = _dev(a, "float32")
        b, pb = _dev(b, b_dtype)
        return True, (a, pa), (b, pb)
    a, pa = _host(a, np.float32)
    b, pb = _host(b, np.dtype(b_dtype))
    return False, (a, pa), (b, pb)


def project(a, b, dt, stream=None):
    """Projected data [2, n_traces] float64 of trace pairs (mg_project): row 0
    <a_i, b_i>_1, row 1 <a_i, b_i>_2."""
    lib = L.load()
    dev, (a, pa), (b, pb) = _traces_pair(a, b, "float32")
    if tuple(a.shape) != tuple(b.shape) or len(a.shape) != 2:
        raise ValueError("a and b must both be [n_traces, nt]")
    R, nt = int(a.shape[0]), int(a.shape[1])
    out = _alloc(dev, (2, R), "float64", a)
    rc = lib.mg_project(pa, pb, R, nt, float(dt), _ptr(out),
                        _stream_ptr(stream) if dev else None, 0 if dev else L.MG_HOST_PTRS)
    L.check(rc, "mg_project")
    return out


def projected_weights(u, z, dt, stream=None):
    """Trace weights [n_traces, nt] float32 (mg_projected_weights) whose
    jacobian_T_apply is the projected-data Jacobian transpose of z [2, n_traces]."""
    lib = L.load()
    dev, (u, pu), (z, pz) = _traces_pair(u, z, "float64")
    R, nt = int(u.shape[0]), int(u.shape[1])
    if tuple(z.shape) != (2, R):
        raise ValueError("z must be [2, n_traces]")
    out = _alloc(dev, (R, nt), "float32", u)
    rc = lib.mg_projected_weights(pu, pz, R, nt, float(dt), _ptr(out),
                                  _stream_ptr(stream) if dev else None,
                                  0 if dev else L.MG_HOST_PTRS)
    L.check(rc, "mg_projected_weights")
    return out


def projected_jacobian_apply(mesh: Mesh, level, eps, shots, wavelet, dt, v, u, nt=None, **kw):
    """Projected Jacobian times v: [2, n_traces] <u_i, (J v)_i>_j."""
    return project(u, jacobian_apply(mesh, level, eps, shots, wavelet, dt, v, nt, **kw), dt)


def projected_jacobian_T_apply(mesh: Mesh, level, eps, shots, wavelet, dt, z, u, nt=None, **kw):
    """Projected Jacobian transpose times z [2, n_traces]: level-cell gradient."""
    return jacobian_T_apply(mesh, level, eps, shots, wavelet, dt, projected_weights(u, z, dt),
                            nt, **kw)


def tv_reconstruct(mesh: Mesh, level_c, eps0, shots, wavelet, dt, dy, *, level_f=-1, u=None,
                   alpha, beta=0.0, n_outer=3, n_cg=50, cg_rtol=1e-8, keep_frac=1.0 / 3.0,
                   ckpt_every=256, nt=None, allow_cfl=False, stream=None):
    """TV-regularised reconstruction (mg_tv_reconstruct): the level-cell
    perturbation x (level_f cells when level_f >= 0, else level_c cells) and
    the per-outer-step history [n_outer, 4] (CG iterations and relative
    residual of the coarse and fine solves).  dy: trace residual [n_traces,
    nt] float32, or projected data [2, n_traces] float64 with the traces u."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    projected = u is not None
    extra = [(dy, "float64" if projected else "float32")]
    if projected:
        extra.append((u, "float32"))
    dev, (eps0, pe), (wav, pw), ex, st, f0 = _prep(eps0, wavelet, extra, stream)
    pdy = ex[0][1]
    pu = ex[1][1] if projected else None
    lev = level_f if level_f >= 0 else level_c
    x = _alloc(dev, (mesh.n_cells_per_level[lev],), "float64", eps0)
    hist = np.zeros((int(n_outer), 4), dtype=np.float64)
    prm = L.mg_tv_params(float(alpha), float(beta), int(n_outer), int(n_cg), float(cg_rtol),
                         float(keep_frac), int(ckpt_every))
    f = f0 | (L.MG_ALLOW_CFL if allow_cfl else 0)
    rc = lib.mg_tv_reconstruct(mesh.handle, int(level_c), int(level_f), pe, C.byref(sh.c), pw,
                               float(dt), nt, L.MG_DATA_PROJECTED if projected else
                               L.MG_DATA_TRACES, pdy, pu, C.byref(prm), _ptr(x),
                               C.c_void_p(hist.ctypes.data), st, f)
    L.check(rc, "mg_tv_reconstruct")
    return x, hist


def tv_reconstruct_levels(mesh: Mesh, levels, eps0, shots, wavelet, dt, dy, *, u=None, alpha,
                          beta=0.0, n_outer=3, n_cg=50, cg_rtol=1e-8, keep_frac=1.0 / 3.0,
                          ckpt_every=256, nt=None, allow_cfl=False, stream=None):
    """Coarse-to-fine reconstruction over the nested ``levels`` (increasing;
    mg_tv_reconstruct_levels): the perturbation x on the cells of the last
    level and the history [n_outer, 2 len(levels)] (CG iterations and
    relative residual of each level's solve, coarse first).  dy, u as in
    tv_reconstruct."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32).ravel())
    projected = u is not None
    extra = [(dy, "float64" if projected else "float32")]
    if projected:
        extra.append((u, "float32"))
    dev, (eps0, pe), (wav, pw), ex, st, f0 = _prep(eps0, wavelet, extra, stream)
    pdy = ex[0][1]
    pu = ex[1][1] if projected else None
    last = int(lv[-1]) if len(lv) else 0
    if not 0 <= last < len(mesh.n_cells_per_level):
        raise ValueError(f"level {last} out of range")
    x = _alloc(dev, (mesh.n_cells_per_level[last],), "float64", eps0)
    hist = np.zeros((int(n_outer), 2 * len(lv)), dtype=np.float64)
    prm = L.mg_tv_params(float(alpha), float(beta), int(n_outer), int(n_cg), float(cg_rtol),
                         float(keep_frac), int(ckpt_every))
    f = f0 | (L.MG_ALLOW_CFL if allow_cfl else 0)
    rc = lib.mg_tv_reconstruct_levels(mesh.handle, C.c_void_p(lv.ctypes.data), len(lv), pe,
                                      C.byref(sh.c), pw, float(dt), nt,
                                      L.MG_DATA_PROJECTED if projected else L.MG_DATA_TRACES,
                                      pdy, pu, C.byref(prm), _ptr(x),
                                      C.c_void_p(hist.ctypes.data), st, f)
    L.check(rc, "mg_tv_reconstruct_levels")
    return x, hist


def approx_jacobian(mesh: Mesh, level, eps, shots, wavelet, dt, u=None, *, want_phi=False,
                    mem_budget=0, nt=None, allow_cfl=False, stream=None):
    """The paper's approximate Jacobian (mg_approx_jacobian).  Returns a dict:
    nodes (caller ids of the level's corner nodes), Lp ([2, n_shots, cells]
    projected columns <u_s, L'_j(s)>_k when u is given) and phi ([n_shots,
    n_nodes, nt] node responses when want_phi)."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    extra = [(u, "float32")] if u is not None else []
    dev, (eps, pe), (wav, pw), ex, st, f0 = _prep(eps, wavelet, extra, stream)
    pu = ex[0][1] if u is not None else None
    n_max = int(mesh.info()["n_nodes"])
    nodes = np.zeros(n_max, dtype=np.int32)
    count = C.c_int64(0)
    f = f0 | (L.MG_ALLOW_CFL if allow_cfl else 0)
    rc = lib.mg_approx_jacobian(mesh.handle, int(level), pe, C.byref(sh.c), pw, float(dt), nt,
                                None, None, None, C.c_void_p(nodes.ctypes.data),
                                C.byref(count), 0, st, f)
    L.check(rc, "mg_approx_jacobian")
    N = int(count.value)
    nl = mesh.n_cells_per_level[level]
    Lp = _alloc(dev, (2, sh.n_shots, nl), "float64", eps) if u is not None else None
    phi = _alloc(dev, (sh.n_shots, N, nt), "float32", eps) if want_phi else None
    if Lp is not None or phi is not None:
        rc = lib.mg_approx_jacobian(mesh.handle, int(level), pe, C.byref(sh.c), pw, float(dt),
                                    nt, pu, _ptr(Lp) if Lp is not None else None,
                                    _ptr(phi) if phi is not None else None, None,
                                    C.byref(count), int(mem_budget), st, f)
        L.check(rc, "mg_approx_jacobian")
    return {"nodes": nodes[:N], "Lp": Lp, "phi": phi}


def forward_pml(mesh: Mesh, eps, shots, wavelet, dt, xi=None, zeta=None, nt=None, *,
                allow_cfl=False, stream=None, flags=0):
    """Traces [n_traces, nt] float32 of the first-order flux leapfrog with the
    split-field layer xi [cells], zeta [cells, dim] (mg_forward_pml); flags
    may add MG_NO_GRAPH."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    extra = [(x, "float64") for x in (xi, zeta) if x is not None]
    dev, (eps, pe), (wav, pw), ex, st, f0 = _prep(eps, wavelet, extra, stream)
    it = iter(ex)
    pxi = next(it)[1] if xi is not None else None
    pzeta = next(it)[1] if zeta is not None else None
    out = _alloc(dev, (sh.n_traces, nt), "float32", eps)
    f = f0 | (L.MG_ALLOW_CFL if allow_cfl else 0) | int(flags)
    rc = lib.mg_forward_pml(mesh.handle, pe, C.byref(sh.c), pw, float(dt), nt, pxi, pzeta,
                            _ptr(out), st, f)
    L.check(rc, "mg_forward_pml")
    return out


def jacobian_apply_pml(mesh: Mesh, level, eps, shots, wavelet, dt, v, xi=None, zeta=None,
                       nt=None, *, allow_cfl=False, stream=None, flags=0):
    """J v [n_traces, nt] float32 of forward_pml's traces for v on the cells of
    ``level`` (mg_jacobian_apply_pml)."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    extra = [(v, "float64")] + [(x, "float64") for x in (xi, zeta) if x is not None]
    dev, (eps, pe), (wav, pw), ex, st, f0 = _prep(eps, wavelet, extra, stream)
    it = iter(ex)
    pv = next(it)[1]
    pxi = next(it)[1] if xi is not None else None
    pzeta = next(it)[1] if zeta is not None else None
    out = _alloc(dev, (sh.n_traces, nt), "float32", eps)
    f = f0 | (L.MG_ALLOW_CFL if allow_cfl else 0) | int(flags)
    rc = lib.mg_jacobian_apply_pml(mesh.handle, int(level), pe, C.byref(sh.c), pw, float(dt),
                                   nt, pxi, pzeta, pv, _ptr(out), st, f)
    L.check(rc, "mg_jacobian_apply_pml")
    return out


def jacobian_T_apply_pml(mesh: Mesh, level, eps, shots, wavelet, dt, w, xi=None, zeta=None,
                         nt=None, *, ckpt_every=64, allow_cfl=False, stream=None, flags=0):
    """J^T w (float64 [cells of level]) of forward_pml's traces for the trace
    weights w [n_traces, nt] float32 (mg_jacobian_T_apply_pml)."""
    lib = L.load()
    sh = Shots.of(shots)
    nt = int(len(wavelet) if nt is None else nt)
    extra = [(w, "float32")] + [(x, "float64") for x in (xi, zeta) if x is not None]
    dev, (eps, pe), (wav, pw), ex, st, f0 = _prep(eps, wavelet, extra, stream)
    it = iter(ex)
    pw_ = next(it)[1]
    pxi = next(it)[1] if xi is not None else None
    pzeta = next(it)[1] if zeta is not None else None
    g = _alloc(dev, (mesh.n_cells_per_level[level],), "float64", eps)
    f = f0 | (L.MG_ALLOW_CFL if allow_cfl else 0) | int(flags)
    rc = lib.mg_jacobian_T_apply_pml(mesh.handle, int(level), pe, C.byref(sh.c), pw, float(dt),
                                     nt, pxi, pzeta, pw_, _ptr(g), int(ckpt_every), st, f)
    L.check(rc, "mg_jacobian_T_apply_pml")
    return g


def _ptr_array(xs):
    return (C.c_void_p * len(xs))(*[C.c_void_p(x.data_ptr() if hasattr(x, "data_ptr")
                                               else x.ctypes.data) for x in xs])


def forward_batch(meshes, eps, shots, wavelets, dts, nt=None, *, allow_cfl=False, stream=None):
    """Traces of several independent problems, one launch per step for all
    (mg_forward_batch).  Returns a list of [n_traces_i, nt] arrays."""
    lib = L.load()
    n = len(meshes)
    sh = [Shots.of(s) for s in shots]
    nt = int(len(wavelets[0]) if nt is None else nt)
    dev = _is_cuda(eps[0])
    if dev:
        ex = [_dev(e, "float64")[0] for e in eps]
        wv = [_dev(x, "float64")[0] for x in wavelets]
        st, f = _stream_ptr(stream), 0
    else:
        ex = [_host(e, np.float64)[0] for e in eps]
        wv = [_host(x, np.float64)[0] for x in wavelets]
        st, f = None, L.MG_HOST_PTRS
    outs = [_alloc(dev, (s.n_traces, nt), "float32", ex[0]) for s in sh]
    shot_arr = (L.mg_shots * n)(*[s.c for s in sh])
    handles = (C.c_void_p * n)(*[m.handle for m in meshes])
    dts_arr = np.ascontiguousarray(dts, dtype=np.float64)
    rc = lib.mg_forward_batch(n, handles, _ptr_array(ex), shot_arr, _ptr_array(wv),
                              C.c_void_p(dts_arr.ctypes.data), nt, _ptr_array(outs), st,
                              f | (L.MG_ALLOW_CFL if allow_cfl else 0))
    L.check(rc, "mg_forward_batch")
    return outs


def jacobian_T_apply_batch(meshes, levels, eps, shots, wavelets, dts, w, nt=None, *,
                           ckpt_every=256, allow_cfl=False, stream=None):
    """J^T w of several independent problems, batched (mg_jacobian_T_apply_batch).
    Returns a list of per-instance level-cell gradients (float64)."""
    lib = L.load()
    n = len(meshes)
    sh = [Shots.of(s) for s in shots]
    nt = int(len(wavelets[0]) if nt is None else nt)
    dev = _is_cuda(eps[0])
    if dev:
        ex = [_dev(e, "float64")[0] for e in eps]
        wv = [_dev(x, "float64")[0] for x in wavelets]
        ww = [_dev(x, "float32")[0] for x in w]
        st, f = _stream_ptr(stream), 0
    else:
        ex = [_host(e, np.float64)[0] for e in eps]
        wv = [_host(x, np.float64)[0] for x in wavelets]
        ww = [_host(x, np.float32)[0] for x in w]
        st, f = None, L.MG_HOST_PTRS
    outs = [_alloc(dev, (m.n_cells_per_level[lv],), "float64", ex[0])
            for m, lv in zip(meshes, levels)]
    shot_arr = (L.mg_shots * n)(*[s.c for s in sh])
    handles = (C.c_void_p * n)(*[m.handle for m in meshes])
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    dts_arr = np.ascontiguousarray(dts, dtype=np.float64)
    rc = lib.mg_jacobian_T_apply_batch(n, handles, C.c_void_p(lv.ctypes.data), _ptr_array(ex),
                                       shot_arr, _ptr_array(wv), C.c_void_p(dts_arr.ctypes.data),
                                       nt, _ptr_array(ww), _ptr_array(outs), int(ckpt_every),
                                       st, f | (L.MG_ALLOW_CFL if allow_cfl else 0))
    L.check(rc, "mg_jacobian_T_apply_batch")
    return outs
