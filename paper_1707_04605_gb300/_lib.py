"""ctypes declarations of the C ABI in include/mgwave.h.

Loading fails loudly (ImportError) when the compiled library is missing:
there is no CPU fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmgwave.so")

MG_OK = 0
MG_ERR_ARG = -1
MG_ERR_NESTING = -2
MG_ERR_OOM = -3
MG_ERR_CUDA = -4
MG_ERR_CFL = -5
MG_ERR_TIMEOUT = -6
MG_ERR_UNSUPPORTED = -7

MG_BC = {"abc": 0, "neumann": 1, "dirichlet": 2}
MG_ORDER = {"rcm": 0, "morton": 1, "none": 2}

MG_HOST_PTRS = 0x01
MG_SINGLE_SOURCE = 0x02
MG_NO_GRAPH = 0x04
MG_PERSISTENT = 0x08
MG_ALLOW_CFL = 0x10
MG_KEEP_CHECKPOINTS = 0x20
MG_REUSE_CHECKPOINTS = 0x40
MG_KEEP_STATES = 0x80


class mg_shots(C.Structure):
    _fields_ = [("n_shots", C.c_int32), ("src", C.POINTER(C.c_int32)),
                ("rec_ptr", C.POINTER(C.c_int64)), ("rec", C.POINTER(C.c_int32))]


MG_DATA_TRACES = 0
MG_DATA_PROJECTED = 1


class mg_tv_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("n_outer", C.c_int),
                ("n_cg", C.c_int), ("cg_rtol", C.c_double), ("keep_frac", C.c_double),
                ("ckpt_every", C.c_int)]


class mg_mesh_info_t(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_levels", C.c_int32), ("n_nodes", C.c_int64),
                ("n_cells", C.c_int64), ("n_bnd", C.c_int64), ("nnz", C.c_int64),
                ("ell_entries", C.c_int64), ("slice_height", C.c_int32),
                ("max_row_nnz", C.c_int32), ("device_bytes", C.c_int64)]


# name -> (restype, argtypes); every symbol include/mgwave.h declares
SIGNATURES = {
    "mg_mesh_create": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "mg_mesh_destroy": (None, [C.c_void_p]),
    "mg_mesh_get_info": (C.c_int, [C.c_void_p, C.POINTER(mg_mesh_info_t)]),
    "mg_mesh_get_permutation": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mg_cfl_dt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                            C.POINTER(C.c_double)]),
    "mg_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(mg_shots), C.c_void_p,
                             C.c_double, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "mg_forward_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(mg_shots), C.c_void_p,
                                     C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_jacobian_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(mg_shots),
                                    C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int]),
    "mg_jacobian_T_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(mg_shots),
                                      C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                      C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "mg_forward_batch": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.POINTER(mg_shots),
                                   C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_int]),
    "mg_jacobian_T_apply_batch": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.POINTER(mg_shots), C.c_void_p, C.c_void_p,
                                            C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                            C.c_void_p, C.c_int]),
    "mg_prolong": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_int]),
    "mg_mesh_set_kernel_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    "mg_mesh_set_shot_groups": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mg_mesh_set_conductivity": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_mesh_set_min_blocks": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_set_kernel_min_blocks": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mg_mesh_set_gather_ring": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mg_mesh_get_gather_ring": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mg_mesh_set_row_sweep": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_get_row_sweep": (C.c_int, [C.c_void_p]),
    "mg_mesh_set_late_prefetch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mg_mesh_set_wide_lanes": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_get_wide_lanes": (C.c_int, [C.c_void_p]),
    "mg_mesh_set_chunked_ell": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_get_late_prefetch": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "mg_mesh_set_tma_tiles": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_set_l1_streaming": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mg_mesh_get_l1_streaming": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mg_mesh_get_tma_tiles": (C.c_int, [C.c_void_p]),
    "mg_mesh_checkpoint_generation": (C.c_int64, [C.c_void_p]),
    "mg_mesh_set_persistent": (C.c_int, [C.c_void_p, C.c_int, C.c_longlong, C.c_int]),
    "mg_mesh_set_bulk_copies": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_set_dependent_launch": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_set_cache_hints": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_set_uniform_ell": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_mesh_device_status": (C.c_int, [C.c_void_p]),
    "mg_tv_reconstruct": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int]),
    "mg_forward_jacobian_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_tv_reconstruct_levels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_int]),
    "mg_approx_jacobian": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_int]),
    "mg_forward_pml": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                 C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int]),
    "mg_jacobian_apply_pml": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int]),
    "mg_jacobian_T_apply_pml": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                          C.c_void_p, C.c_int]),
    "mg_project": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double,
                             C.c_void_p, C.c_void_p, C.c_int]),
    "mg_projected_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                       C.c_double, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_mesh_get_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mg_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(mg_shots), C.c_void_p,
                              C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "mg_mesh_trim": (C.c_int, [C.c_void_p]),
    "mg_mesh_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    "mg_launch_count": (C.c_int64, [C.c_void_p]),
    "mg_strerror": (C.c_char_p, [C.c_int]),
    "mg_version": (C.c_int, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library and declare every entry point; raises ImportError
    if the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library not built: {path} is missing "
            "(run paper_1707_04605_gb300.build.build() first)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MgError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().mg_strerror(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def check(code: int, where: str):
    if code != MG_OK:
        raise MgError(code, where)
