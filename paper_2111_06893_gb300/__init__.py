"""GB300 (sm_103a) library for DG models of Brownian coating thermal noise.

The compute path is the CUDA library libthermonoise.so (C ABI in
include/thermonoise.h); ``thermonoise`` is its thin Python binding.
"""
from . import thermonoise
from .thermonoise import Context, noise_psd, setup

__all__ = ["thermonoise", "Context", "noise_psd", "setup"]
