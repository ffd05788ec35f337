"""B300-native solver for the effective thermal conductivity of voxel RVEs.

Hot path of Ye, Fu & Chung (arXiv 2404.02433): TPFA discretisation, PCG with
a homogeneous-reference preconditioner inverted by cosine transforms and
tridiagonal solves, outflow-flux ETC.  The computation lives in libetc.so
(CUDA, sm_103a) behind a C ABI (include/etc.h); ``binding`` marshals
arguments to it (``from paper_2404_02433_b300 import binding``).
``microstructure`` holds seeded input generators.
"""
from . import microstructure  # noqa: F401

__all__ = ["microstructure", "binding"]
