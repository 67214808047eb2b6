"""GB300-native (sm_103a) RLT2 Lagrangian dual ascent for QAP lower bounds.

The compute path is the CUDA library ``librlt2.so`` (C ABI: include/rlt2.h);
``rlt2`` is its ctypes binding and ``instances`` the seeded synthetic inputs.
Importing the package does not load the library; the first call does, and it
fails loudly if the library has not been built.
"""
from . import instances  # noqa: F401

__all__ = ["instances", "rlt2", "build"]
