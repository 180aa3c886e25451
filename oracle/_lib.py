"""Builds and loads oracle.c (plain C, gcc, OpenMP).  Test infrastructure only."""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (no -march flags: same on x86 and Arm)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        P = ctypes.c_void_p
        L.or_direct_sum.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_long, P, P, P, P,
                                    ctypes.c_long, P, P, P, P]
        L.or_direct_sum.restype = None
        L.or_tri_sl.argtypes = [P, P, P, P]
        L.or_tri_sl.restype = ctypes.c_double
        L.or_tri_dl.argtypes = [P, P, P, P]
        L.or_tri_dl.restype = ctypes.c_double
        L.or_assemble_p0.argtypes = [ctypes.c_long, P, ctypes.c_long, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P]
        L.or_assemble_p0.restype = ctypes.c_int
        L.or_regular_rule.argtypes = [ctypes.c_int, P, P]
        L.or_regular_rule.restype = ctypes.c_int
        L.or_triangle_rule.argtypes = [ctypes.c_int, P, P, P]
        L.or_triangle_rule.restype = None
        L.or_tri_lin.argtypes = [P, P, P, P, P, P]
        L.or_tri_lin.restype = None
        L.or_assemble_p1.argtypes = [ctypes.c_long, P, ctypes.c_long, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
        L.or_assemble_p1.restype = ctypes.c_int
        L.or_pair_p1.argtypes = [P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, P]
        L.or_pair_p1.restype = ctypes.c_int
        L.or_corrections_p0.argtypes = [ctypes.c_long, P, ctypes.c_long, P, ctypes.c_long, P, P, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.or_corrections_p0.restype = ctypes.c_int
        _lib = L
    return _lib
