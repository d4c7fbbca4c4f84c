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
    mg, L, lib = env
    w = configs.asteroid_2d(n_refine=2, S=37, nt=400)
    mesh = mg.mesh_from_workload(w)
    dt = oracle_dt(w)
    eps = torch.as_tensor(w.eps, dtype=torch.float64, device="cuda")
    wav = torch.as_tensor(w.wavelet(dt), dtype=torch.float64, device="cuda")
    ref = mg.forward(mesh, eps, w.shots, wav, dt).cpu().numpy()
    shots = mg.Shots.of(w.shots)
    outs = [torch.full((shots.n_traces, w.nt), np.nan, dtype=torch.float32, device="cuda")
            for _ in range(2)]
    torch.cuda.synchronize()
    for i, out in enumerate(outs):
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call(lib, L, mesh, eps, shots, wav, dt, w.nt, out)
        torch.cuda.synchronize()
        assert rc == L.MG_OK, lib.mg_strerror(rc)
        if i == 1:
            # no device memory was reserved by the call
            assert torch.cuda.mem_get_info()[0] == free_before
        y = out.cpu().numpy()
        assert np.isfinite(y).all()
        assert rel_l2(y, ref) < TRACE_TOL


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
