"""GB300-native CLoD-GS rasterizer: continuous level of detail for 3D Gaussian
splatting (distance-decay opacity, dynamic-threshold cull, tile-based
depth-sorted alpha blending, hand-written backward), behind the C ABI of
include/clod.h.

Submodules are imported on demand so that the synthetic-input generator
(``synth``) can be used without a GPU or the compiled library.
"""
__all__ = ["synth", "clod", "autograd", "train", "serve", "abi"]
