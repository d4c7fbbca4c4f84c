"""torch.autograd.Function over the library's forward and adjoint.

traces(dc) = forward(eps0 + P dc): dc holds a permittivity perturbation per
cell of a coarse level of the nested mesh (Sec. II-B, eps_r = sum_j c_j
chi'_j), P is the nested prolongation to the finest cells.  The forward
keeps checkpoints on the mesh handle; the backward applies J^T to the
incoming trace gradient with the discrete adjoint, reusing those checkpoints
when the handle still holds them (otherwise it recomputes them).  Every
numeric step runs in the CUDA library; this module only routes tensors.
"""
from __future__ import annotations

import torch

from . import _lib as L
from . import api


class LevelTraces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dc, mesh, level, eps0, shots, wavelet, dt, ckpt_every):
        eps = api.prolong(mesh, level, dc.detach().contiguous(), eps0)
        y = api.forward(mesh, eps, shots, wavelet, dt, ckpt_every=ckpt_every,
                        keep_checkpoints=True)
        ctx.save_for_backward(eps, wavelet)
        ctx.meta = (mesh, level, shots, dt, ckpt_every)
        return y

    @staticmethod
    def backward(ctx, gy):
        eps, wavelet = ctx.saved_tensors
        mesh, level, shots, dt, ckpt_every = ctx.meta
        w = gy.detach().to(torch.float32).contiguous()
        try:
            g = api.jacobian_T_apply(mesh, level, eps, shots, wavelet, dt, w,
                                     ckpt_every=ckpt_every, reuse_checkpoints=True)
        except L.MgError as e:
            if e.code != L.MG_ERR_ARG:
                raise
            g = api.jacobian_T_apply(mesh, level, eps, shots, wavelet, dt, w,
                                     ckpt_every=ckpt_every)
        return g, None, None, None, None, None, None, None


def level_traces(dc, mesh, level, eps0, shots, wavelet, dt, ckpt_every=256):
    """Differentiable traces [n_traces, nt] of the level-cell perturbation dc
    (CUDA float64 [cells of level]); eps0, wavelet: CUDA float64."""
    return LevelTraces.apply(dc, mesh, level, eps0, shots, wavelet, dt, ckpt_every)
