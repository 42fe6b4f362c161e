"""Seeded synthetic inputs (meshes and initial states) shared by the oracle and the CUDA path.

Nothing here computes any part of the scheme; see ``voronoi`` and ``states``.
"""
