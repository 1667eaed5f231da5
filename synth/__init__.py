"""Seeded synthetic inputs (meshes, features, ground truth) shared by the oracle and the CUDA path.

Holds no part of the matching method itself."""
from . import instances, meshes  # noqa: F401
