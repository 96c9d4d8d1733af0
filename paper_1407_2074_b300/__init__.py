"""B300-native multi-channel octree ray caster (Brix, Prassni, Hinrichs, arXiv 1407.2074).

The compute path is libvr.so (hand-written sm_103a CUDA behind the C ABI in include/vr.h);
this package only marshals arguments to it.
"""
from .vr import Renderer, RenderFn, render, VRError, LIB_PATH  # noqa: F401
from . import dist  # noqa: F401
