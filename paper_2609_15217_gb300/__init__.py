"""GB300-native tiny batched LU with partial pivoting (n <= 32) and a fused
per-point Newton kernel.

The compute path is the CUDA shared library built from csrc/ (C ABI declared
in include/tinylu.h); `tinylu` is its thin ctypes binding.  Importing this
package does not load the library: `paper_2609_15217_gb300.tinylu` does, and
it raises if the library is missing (there is no CPU fallback).
"""
__all__ = ["inputs", "tinylu", "build"]
