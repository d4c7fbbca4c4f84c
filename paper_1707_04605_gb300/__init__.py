"""GB300-native leapfrog wave propagation and exact Jacobian on nested P1
meshes (Takala, Us, Pursiainen: multigrid-based radar tomography).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/mgwave.h``); this package only marshals arguments to it.
"""
from . import _lib  # noqa: F401
from .api import (Mesh, Shots, cfl_dt, forward, forward_batch,  # noqa: F401
                  jacobian_T_apply, jacobian_T_apply_batch, jacobian_apply, mesh_create,
                  mesh_from_workload, project, projected_jacobian_T_apply,
                  projected_jacobian_apply, projected_weights, prolong, tv_reconstruct,
                  tv_reconstruct_levels, approx_jacobian, forward_pml, jacobian_apply_pml,
                  forward_jacobian_apply,
                  jacobian_T_apply_pml)

__all__ = ["Mesh", "Shots", "mesh_create", "mesh_from_workload", "cfl_dt", "forward",
           "jacobian_apply", "jacobian_T_apply", "forward_batch", "jacobian_T_apply_batch",
           "prolong", "project", "projected_weights", "projected_jacobian_apply",
           "projected_jacobian_T_apply", "tv_reconstruct", "tv_reconstruct_levels",
           "approx_jacobian",
           "forward_pml", "jacobian_apply_pml", "jacobian_T_apply_pml",
           "forward_jacobian_apply"]
