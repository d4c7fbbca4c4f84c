"""mg_forward_noalloc: the forward for callers that cannot let the library
allocate (their own memory pool owns the device, or an allocation and its
implicit synchronisation is not allowed where they call).  The entry point
uses only a fixed device array compiled into the library; this test calls it
through the C ABI and checks it against mg_forward, twice in a row (the
array keeps the previous call's contents, so the second call checks that
everything that must start at zero is cleared), and that it reserves no
device memory while it runs.

This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import TRACE_TOL, oracle_dt, rel_l2
from workloads import configs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env(cuda_device):
    from paper_1707_04605_gb300 import build

    build.build()
    import paper_1707_04605_gb300 as mg
    from paper_1707_04605_gb300 import _lib as L

    return mg, L, L.load()


def _call(lib, L, mesh, eps, shots, wav, dt, nt, out, flags=0):
    sh = shots.c
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.mg_forward_noalloc(mesh.handle, C.c_void_p(eps.data_ptr()), C.byref(sh),
                                  C.c_void_p(wav.data_ptr()), float(dt), int(nt),
                                  C.c_void_p(out.data_ptr()), stream, flags)


def test_noalloc_forward_matches_forward_twice(env):
    """Two calls in a row with different inputs: the second has another
    permittivity, fewer shots at other nodes with other receivers, and a
    shorter run, so contents the first call left in the shared array
    (coefficients, event lists, the FP32 wavelet) would show in its traces.
    Neither call changes the device's free memory: the array was reserved
    when the mesh handle was created."""
    mg, L, lib = env
    w = configs.asteroid_2d(n_refine=2, S=37, nt=400)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    cases = []
    for eps_h, sh, nt in ((w.eps, w.shots, w.nt),
                          (w.eps * np.where(np.arange(len(w.eps)) % 3 == 0, 1.1, 1.0),
                           configs.asteroid_2d(n_refine=2, S=12, rotation=0.3).shots, 250)):
        eps = torch.as_tensor(eps_h, dtype=torch.float64, device="cuda")
        wav = torch.as_tensor(w.wavelet(dt, nt), dtype=torch.float64, device="cuda")
        ref = mg.forward(mesh, eps, sh, wav, dt).cpu().numpy()
        cases.append((eps, mg.Shots.of(sh), wav, nt, ref))
    assert cases[1][1].n_traces != cases[0][1].n_traces
    torch.cuda.synchronize()
    for eps, shots, wav, nt, ref in cases:
        out = torch.full((shots.n_traces, nt), np.nan, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call(lib, L, mesh, eps, shots, wav, dt, nt, out)
        torch.cuda.synchronize()
        assert rc == L.MG_OK, lib.mg_strerror(rc)
        assert torch.cuda.mem_get_info()[0] == free_before
        y = out.cpu().numpy()
        assert np.isfinite(y).all()
        assert rel_l2(y, ref) < TRACE_TOL
    # dt above the stability bound is refused unless MG_ALLOW_CFL is given
    eps, shots, wav, nt, _ = cases[0]
    out = torch.zeros((shots.n_traces, nt), dtype=torch.float32, device="cuda")
    dt_big = 1.01 * mg.cfl_dt(mesh, eps)
    assert _call(lib, L, mesh, eps, shots, wav, dt_big, nt, out) == L.MG_ERR_CFL


def test_noalloc_rejects_work_beyond_its_array(env):
    mg, L, lib = env
    w = configs.asteroid_2d(n_refine=3, S=256, nt=10)   # 2 x 62,641 x 256 x 4 B > 64 MiB
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    eps = torch.as_tensor(w.eps, dtype=torch.float64, device="cuda")
    wav = torch.as_tensor(w.wavelet(dt), dtype=torch.float64, device="cuda")
    shots = mg.Shots.of(w.shots)
    out = torch.zeros((shots.n_traces, w.nt), dtype=torch.float32, device="cuda")
    assert _call(lib, L, mesh, eps, shots, wav, dt, w.nt, out) == L.MG_ERR_ARG
    assert _call(lib, L, mesh, eps, shots, wav, dt, w.nt, out, flags=L.MG_KEEP_CHECKPOINTS) \
        == L.MG_ERR_UNSUPPORTED
