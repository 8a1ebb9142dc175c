"""GB300-native voxel-grid decimation of point clouds (arXiv 2102.11084).

The compute path is the CUDA library ``libvg.so`` behind the C ABI in
``include/vg.h``; ``vg`` is its Python binding.  ``synth`` makes seeded test clouds.
"""
from .vg import (Decimation, Status, VGError, downsample, downsample_into, alloc_buffers,  # noqa: F401
                 workspace_bytes, version, lib)

__all__ = ["Decimation", "Status", "VGError", "downsample", "downsample_into", "alloc_buffers",
           "workspace_bytes", "version", "lib"]
