"""Build and load the oracle's C library (oracle.c) with gcc + OpenMP.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_handle = None


def build(force=False):
    """Compile oracle.c into oracle/_build/liboracle.so (portable flags only).

    -ffp-contract=off keeps a*b+c as two roundings on every host (aarch64 GCC
    would otherwise fuse them), so the oracle rounds the same way on x86 and Arm.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _handle
    with _lock:
        if _handle is None:
            path = build()
            h = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            h.oracle_jacobi_eig.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_double]
            h.oracle_jacobi_eig.restype = ctypes.c_int
            h.oracle_efloat_scan.argtypes = [ctypes.c_int, dp, dp, dp]
            h.oracle_efloat_scan.restype = None
            h.oracle_num_threads.argtypes = []
            h.oracle_num_threads.restype = ctypes.c_int
            _handle = h
        return _handle


def dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
