"""GB300-native hot path of the Accessibility Field method (arxiv 2608.06412).

Scan-centric TSDF integration into a sparse voxel-brick hash, a bit-packed
occupied / known view, and per-surface-point accessibility scoring against
precomputed tool and corridor voxel kernels, as hand-written sm_103a CUDA
behind the C ABI of include/af.h.

Submodules (imported on demand, so that importing the package needs neither
a GPU nor the compiled library):
  af     -- the Python binding of libaf (Map, MapConfig, ToolConfig, ...)
  build  -- compiles libaf.so in-tree with nvcc
  synth  -- seeded synthetic scans, scenes and direction tables
"""
__all__ = ["af", "build", "synth"]
