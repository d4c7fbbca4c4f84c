"""The C-ABI library builds, loads and exports every symbol the header
declares; host-side argument checks run before any CUDA call (no GPU)."""
import ctypes as C
import re

import numpy as np
import pytest

from paper_1707_04605_gb300 import _lib as L
from paper_1707_04605_gb300 import api, build
from workloads import configs, meshes

HEADER = build.INCLUDE + "/mgwave.h"


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(mg_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in L.SIGNATURES, f"{name} missing from the binding"
    assert set(L.SIGNATURES) == set(names)


def test_error_strings(lib):
    assert lib.mg_strerror(0) == b"ok"
    for code in range(-7, 0):
        assert lib.mg_strerror(code) not in (b"ok", b"unknown error")
    assert lib.mg_strerror(-100) == b"unknown error"
    assert lib.mg_version() >= 100


def _create(lib, m, **over):
    args = dict(dim=m.dim, coords=m.coords, cells=m.cells, parents=m.cell_parent,
                ncl=m.n_cells, bnd=m.bnd, bc=0, order=0)
    args.update(over)
    coords = np.ascontiguousarray(args["coords"], np.float64)
    cells = np.ascontiguousarray(args["cells"], np.int32)
    bnd = np.ascontiguousarray(args["bnd"], np.int32)
    ncl = np.ascontiguousarray(args["ncl"], np.int64)
    pars = [np.ascontiguousarray(p, np.int32) for p in args["parents"]]
    arr = (C.c_void_p * max(1, len(pars)))(*[p.ctypes.data for p in pars])
    h = C.c_void_p()
    rc = lib.mg_mesh_create(args["dim"], len(ncl), coords.ctypes.data, coords.shape[0],
                            cells.ctypes.data, cells.shape[0],
                            C.cast(arr, C.c_void_p) if pars else None, ncl.ctypes.data,
                            bnd.ctypes.data, bnd.shape[0], args["bc"], args["order"],
                            C.byref(h))
    if rc == 0:
        lib.mg_mesh_destroy(h)
    return rc


@pytest.mark.parametrize("case,code", [
    ("dim", L.MG_ERR_ARG),
    ("cell_range", L.MG_ERR_ARG),
    ("repeated_node", L.MG_ERR_ARG),
    ("degenerate", L.MG_ERR_ARG),
    ("unused_node", L.MG_ERR_ARG),
    ("facet_not_on_cell", L.MG_ERR_ARG),
    ("parent_range", L.MG_ERR_NESTING),
    ("childless_parent", L.MG_ERR_NESTING),
    ("level_count", L.MG_ERR_ARG),
    ("bc", L.MG_ERR_ARG),
    ("nan_coord", L.MG_ERR_ARG),
])
def test_invalid_meshes_rejected_before_cuda(lib, case, code):
    m = meshes.square_mesh(2, 1)
    cells = m.cells.copy()
    coords = m.coords.copy()
    parents = [p.copy() for p in m.cell_parent]
    ncl = list(m.n_cells)
    bnd = m.bnd.copy()
    over = {}
    if case == "dim":
        over["dim"] = 4
    elif case == "cell_range":
        cells[3, 1] = len(coords)
    elif case == "repeated_node":
        cells[0, 1] = cells[0, 0]
    elif case == "degenerate":
        coords[cells[0, 2]] = 0.5 * (coords[cells[0, 0]] + coords[cells[0, 1]])
    elif case == "unused_node":
        coords = np.concatenate([coords, [[5.0, 5.0]]])
    elif case == "facet_not_on_cell":
        bnd[0] = [cells[0, 0], cells[5, 2]] if cells[0, 0] != cells[5, 2] else [0, 7]
    elif case == "parent_range":
        parents[0][0] = ncl[0]
    elif case == "childless_parent":
        parents[0][parents[0] == 1] = 0
    elif case == "level_count":
        ncl[-1] += 1
    elif case == "bc":
        over["bc"] = 7
    elif case == "nan_coord":
        coords[0, 0] = np.nan
    over.update(coords=coords, cells=cells, parents=parents, ncl=ncl, bnd=bnd)
    assert _create(lib, m, **over) == code


def test_valid_mesh_reaches_the_device_step(lib):
    """A valid mesh passes every host check; without a GPU the first CUDA
    call fails with MG_ERR_CUDA, with one the handle is created."""
    m = meshes.square_mesh(2, 1)
    rc = _create(lib, m)
    assert rc in (L.MG_OK, L.MG_ERR_CUDA)


def test_binding_refuses_missing_library(tmp_path):
    saved = L._lib
    try:
        L._lib = None
        with pytest.raises(ImportError):
            L.load(str(tmp_path / "missing.so"))
    finally:
        L._lib = saved


def test_shots_marshalling():
    w = configs.tiny_2d()
    sh = api.Shots.of(w.shots)
    assert sh.c.n_shots == w.shots.n_shots
    assert sh.n_traces == w.shots.n_traces
    assert sh.c.src[0] == w.shots.src[0]
    assert sh.c.rec_ptr[sh.n_shots] == w.shots.rec_ptr[-1]
