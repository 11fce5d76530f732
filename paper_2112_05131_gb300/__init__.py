"""Plenoxels differentiable sparse-voxel renderer (arXiv 2112.05131) for GB300 (sm_103a).

All computation runs in libplenoxel (CUDA, C ABI in include/plenoxel.h); this
package allocates device memory with PyTorch and marshals arguments.
"""
from ._lib import PLX_SH_BF16, PLX_SH_F32, PlxError, load  # noqa: F401

__all__ = ["PLX_SH_F32", "PLX_SH_BF16", "PlxError", "load"]
