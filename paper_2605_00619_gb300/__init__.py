"""GB300-native quadrature-free ADER-AFE-DG step on 3D polyhedral meshes.

The compute path lives in the C-ABI library ``lib/libafe.so`` (CUDA kernels for sm_103a,
declared in ``include/afe.h``); :mod:`paper_2605_00619_gb300.afe` is its thin Python
binding and :mod:`paper_2605_00619_gb300.build` compiles it in-tree.
"""
from . import afe  # noqa: F401
