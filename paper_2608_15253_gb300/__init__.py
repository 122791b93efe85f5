"""GB300-native (sm_103a) micromagnetic LLG hot path of arxiv 2608.15253.

The compute path lives in ``libmm.so`` (CUDA kernels behind the C ABI in
``include/mm.h``).  This package is the thin Python binding over that ABI:
``mm`` mirrors every C function under the same name and only marshals
arguments (numpy arrays, torch tensors' device pointers).  It fails loudly
when the library is missing; there is no CPU fallback.
"""
from .mm import *  # noqa: F401,F403
from .mm import lib_path, load, MMError  # noqa: F401
