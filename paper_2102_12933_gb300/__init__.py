"""GB300-native residual and SSP-RK3 stage of the unstructured-mesh FDM.

Zhen, Qu & Cai, "A Novel Finite Difference Method for Euler Equations in
2D Unstructured Meshes" (arXiv 2102.12933).  The compute path is the
C-ABI library ``libfdu.so`` (hand-written CUDA for sm_103a) declared in
``include/fdu.h``; :mod:`paper_2102_12933_gb300.fdu` is its thin Python
binding.  The binding loads the library lazily, so importing this package
(for example for :mod:`paper_2102_12933_gb300.inputs`) needs no GPU.
"""
__all__ = ["inputs", "fdu"]
