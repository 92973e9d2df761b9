"""GB300 (sm_103a) Huffman decoding of error-bounded lossy compression codes.

The decode path lives in libhd.so (C ABI in include/hd.h, CUDA kernels in
csrc/); ``hd`` is its thin ctypes binding.
"""
from . import build
from .hd import (Context, DeviceField, HDError, hd_build_codebook, hd_encode, hd_version, load,
                 library_path)

__all__ = ["build", "Context", "DeviceField", "HDError", "hd_build_codebook", "hd_encode",
           "hd_version", "load", "library_path"]
