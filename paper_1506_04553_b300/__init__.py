"""paper_1506_04553_b300 -- the tree side of the P3T scheme (Iwasawa,
Portegies Zwart & Makino, arXiv:1506.04553) on one NVIDIA B300.

The compute path is libp3t.so (hand-written CUDA for sm_103a behind the C ABI
of include/p3t.h); ``binding`` is its thin ctypes wrapper, loaded on first
use of any of the names below (it raises if the library cannot be loaded:
there is no CPU fallback).  ``ics`` holds the seeded initial-condition
generators and needs no GPU.
"""
from __future__ import annotations

_BINDING_NAMES = {"Params", "Context", "P3TError", "kick", "drift",
                  "library_path", "launch_count", "alu_peaks", "FLAG_NO_SYNC",
                  "HermiteParams", "hard_force", "fp64_peaks"}

__all__ = sorted(_BINDING_NAMES) + ["ics", "binding"]


def __getattr__(name):
    if name in _BINDING_NAMES or name == "binding":
        import importlib
        mod = importlib.import_module(__name__ + ".binding")
        return mod if name == "binding" else getattr(mod, name)
    raise AttributeError(name)
