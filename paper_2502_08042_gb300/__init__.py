"""GB300-native exact k-core decomposition by parallel peeling (arXiv 2502.08042).

The compute runs in libkcore.so (hand-written CUDA for sm_103a behind the C ABI
of include/kcore.h); this package only builds/loads it and marshals arguments.
"""
from ._native import build, lib  # noqa: F401
from .kcore import KCore, KCoreError, KCoreServer, decompose  # noqa: F401

__all__ = ["build", "lib", "KCore", "KCoreError", "KCoreServer", "decompose"]
