"""Builds tests/user_kernels.c (gcc) and hands its functions out as ctypes function
pointers with their parameter blocks, for the solver's and the oracle's user-kernel
interfaces."""
from __future__ import annotations

import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "user_kernels.c")
LIB = os.path.join(HERE, "_build", "libuserkernels.so")
_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            tmp = LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"], check=True)
            os.replace(tmp, LIB)
        _lib = ctypes.CDLL(LIB)
        for name in ("hpm_test_erf_g", "hpm_test_erf_dg", "hpm_test_plummer_g", "hpm_test_plummer_dg"):
            fn = getattr(_lib, name)
            fn.argtypes = [ctypes.c_double, ctypes.c_void_p]
            fn.restype = ctypes.c_double
    return _lib


class Param:
    """A double the kernel reads through its ctx pointer (kept alive with this object)."""

    def __init__(self, value: float):
        self.v = ctypes.c_double(value)

    @property
    def ptr(self):
        return ctypes.cast(ctypes.pointer(self.v), ctypes.c_void_p)


def erf_kernel(a: float):
    """(g, dg, param) of erf(r/a)/r."""
    L = lib()
    return L.hpm_test_erf_g, L.hpm_test_erf_dg, Param(a)


def plummer_kernel(eps: float):
    L = lib()
    return L.hpm_test_plummer_g, L.hpm_test_plummer_dg, Param(eps)
