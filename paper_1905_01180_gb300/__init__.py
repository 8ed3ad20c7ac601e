"""GB300-native GKBA second-Born collision integral (arXiv:1905.01180).

The compute path lives in the C-ABI library libgkba.so (include/gkba.h,
CUDA kernels for sm_103a under csrc/); ``gkba`` is its Python binding.
"""
from .gkba import Batch, Context, GKBAError, load, FP64, SPLIT_TF32, SPLIT_TF32_ACC  # noqa: F401
