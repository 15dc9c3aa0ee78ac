"""GB300-native fused streaming + MRT collision step of the iD3Q14 / iD3Q18
incompressible lattice Boltzmann models (arXiv:1503.03337).

The compute path is the CUDA library ``liblbm.so`` (C-ABI in include/lbm.h);
``lbm`` is its ctypes binding.
"""
from . import lbm  # noqa: F401
