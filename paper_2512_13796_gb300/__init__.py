"""Nexels image formation (neurally-textured surfels) on one GB300.

The rendering path is libnexel.so (CUDA kernels for sm_103a behind the C ABI
in include/nexel.h); this package builds it, binds it with ctypes and wraps
it in a torch.autograd.Function.
"""
from . import synth  # noqa: F401
from ._native import build, lib  # noqa: F401

__all__ = ["build", "lib", "synth"]
