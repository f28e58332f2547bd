"""Host build of the device header's draw rounding for the CPU tests (a
test-side tool, not part of the library): nvcc compiles grid_host.cu as
host code against the library's own table builder."""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(os.path.dirname(_HERE))
_SRC = os.path.join(_HERE, "grid_host.cu")
_DEPS = [_SRC, os.path.join(_ROOT, "paper_2108_05815_b300", "csrc", "device.cuh"),
         os.path.join(_ROOT, "paper_2108_05815_b300", "csrc", "tables.cpp")]
_LIB = os.path.join(_HERE, "_build", "libgridhost.so")


def build():
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not os.path.exists(_LIB) or any(os.path.getmtime(p) > os.path.getmtime(_LIB) for p in _DEPS):
        nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.run([nvcc if os.path.exists(nvcc) else "nvcc", "-std=c++17", "-O2",
                        "-Xcompiler", "-fPIC", "-shared", _SRC, _DEPS[2], "-lquadmath", "-o", tmp],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.grid_draws.restype = ctypes.c_int
        L.grid_draws.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]
        _lib = L
    return _lib


def grid_draws(r, sft):
    """(x58, a, near) arrays of the header's exp1_grid for r53 values and grid shifts"""
    import numpy as np
    r = np.ascontiguousarray(r, dtype=np.uint64)
    sft = np.ascontiguousarray(sft, dtype=np.int32)
    n = len(r)
    x58 = np.zeros(n, dtype=np.uint64)
    a = np.zeros(n, dtype=np.uint64)
    near = np.zeros(n, dtype=np.uint8)
    rc = lib().grid_draws(r.ctypes.data, sft.ctypes.data, n, x58.ctypes.data, a.ctypes.data, near.ctypes.data)
    if rc != 0:
        raise ValueError("grid_draws: argument out of range")
    return x58, a, near.astype(bool)
