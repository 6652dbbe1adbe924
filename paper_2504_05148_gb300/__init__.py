"""GB300 (sm_103a) stereo-LiDAR semi-global matching.

The CUDA library ``lib/libsgmf.so`` (built by ``build.py`` from ``csrc/``)
computes the pipeline of Yao et al., "Stereo-LiDAR Fusion by Semi-Global
Matching with Discrete Disparity-Matching Cost and Semidensification"
(RA-L 2025, Fig. 1) behind the C ABI of ``include/sgmf.h``; ``sgmf`` is its
ctypes binding and ``scenes`` the seeded synthetic input generator.
"""
from . import sgmf  # noqa: F401
from .sgmf import Context, Params  # noqa: F401
