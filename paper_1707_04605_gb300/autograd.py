"""torch.autograd.Function over the library's forward and adjoint.

traces(dc) = forward(eps0 + P dc): dc holds a permittivity perturbation per
cell of a coarse level of the nested mesh (Sec. II-B, eps_r = sum_j c_j
chi'_j), P is the nested prolongation to the finest cells.  The forward
keeps checkpoints on the mesh handle and records the handle's checkpoint
generation; the backward applies J^T to the incoming trace gradient with
the discrete adjoint, reusing those checkpoints only while the generation is
unchanged (no other call has rewritten them, e.g. a second forward with
another perturbation), otherwise recomputing them.  Every numeric step runs
in the CUDA library; this module only routes tensors.
"""
from __future__ import annotations

import torch

from . import api


class LevelTraces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dc, mesh, level, eps0, shots, wavelet, dt, ckpt_every):
        eps = api.prolong(mesh, level, dc.detach().contiguous(), eps0)
        y = api.forward(mesh, eps, shots, wavelet, dt, ckpt_every=ckpt_every,
                        keep_checkpoints=True)
        ctx.save_for_backward(eps, wavelet)
        ctx.meta = (mesh, level, shots, dt, ckpt_every, mesh.checkpoint_generation())
        return y

    @staticmethod
    def backward(ctx, gy):
        eps, wavelet = ctx.saved_tensors
        mesh, level, shots, dt, ckpt_every, gen = ctx.meta
        w = gy.detach().to(torch.float32).contiguous()
        reuse = mesh.checkpoint_generation() == gen
        g = api.jacobian_T_apply(mesh, level, eps, shots, wavelet, dt, w,
                                 ckpt_every=ckpt_every, reuse_checkpoints=reuse)
        return g, None, None, None, None, None, None, None


def level_traces(dc, mesh, level, eps0, shots, wavelet, dt, ckpt_every=256):
    """Differentiable traces [n_traces, nt] of the level-cell perturbation dc
    (CUDA float64 [cells of level]); eps0, wavelet: CUDA float64."""
    return LevelTraces.apply(dc, mesh, level, eps0, shots, wavelet, dt, ckpt_every)
