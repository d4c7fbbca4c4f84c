"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Meshes, permittivity fields, shot geometry and source wavelets only; nothing
here computes any part of the wave scheme or its derivatives.
"""
from . import configs, fields, meshes, shots  # noqa: F401
