"""ctypes binding of oracle_core.c (test infrastructure only; see package doc).

``build()`` compiles the C core with gcc (plain -O2, OpenMP over outer loops).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_core.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i32, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        P = ctypes.c_void_p
        L.orc_gauss_legendre01.argtypes = [i32, P, P]
        L.orc_dunavant6.argtypes = [P, P]
        L.orc_rule_far.argtypes = [P, P, i32, i32]
        L.orc_rule_far.restype = d
        L.orc_rule_identical.argtypes = [P, i32, i32]
        L.orc_rule_identical.restype = d
        L.orc_rule_edge.argtypes = [P, P, i32, i32]
        L.orc_rule_edge.restype = d
        L.orc_rule_vertex.argtypes = [P, P, i32, i32]
        L.orc_rule_vertex.restype = d
        L.orc_assemble_V.argtypes = [i64, P, P, i32, i32, P]
        L.orc_V_entries.argtypes = [i64, P, P, P, P, i32, i32, P]
        L.orc_pair_kernel.argtypes = [P, P, i64, i64, i32, i32, i32]
        L.orc_pair_kernel.restype = d
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def gauss_legendre01(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_legendre01(n, _p(x), _p(w)) != 0:
        raise ValueError(n)
    return x, w


def dunavant6():
    b = np.zeros((6, 3))
    w = np.zeros(6)
    lib().orc_dunavant6(_p(b), _p(w))
    return b, w


def rule_far(P, Q, kernel=0, far_order=0) -> float:
    P = np.ascontiguousarray(P, float)
    Q = np.ascontiguousarray(Q, float)
    return lib().orc_rule_far(_p(P), _p(Q), kernel, far_order)


def rule_identical(P, n=5, kernel=0) -> float:
    P = np.ascontiguousarray(P, float)
    return lib().orc_rule_identical(_p(P), n, kernel)


def rule_edge(P, Q, n=5, kernel=0) -> float:
    P = np.ascontiguousarray(P, float)
    Q = np.ascontiguousarray(Q, float)
    return lib().orc_rule_edge(_p(P), _p(Q), n, kernel)


def rule_vertex(P, Q, n=5, kernel=0) -> float:
    P = np.ascontiguousarray(P, float)
    Q = np.ascontiguousarray(Q, float)
    return lib().orc_rule_vertex(_p(P), _p(Q), n, kernel)


def pair(xyz, tri, T, S, far_order=0, ss_order=5, kernel=0) -> float:
    xyz = np.ascontiguousarray(xyz, float)
    tri = np.ascontiguousarray(tri, np.int32)
    return lib().orc_pair_kernel(_p(xyz), _p(tri), int(T), int(S), far_order, ss_order, kernel)


def assemble_V(xyz, tri, far_order=0, ss_order=5) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, float)
    tri = np.ascontiguousarray(tri, np.int32)
    nt = tri.shape[0]
    V = np.empty((nt, nt), dtype=np.float64)
    lib().orc_assemble_V(nt, _p(xyz), _p(tri), far_order, ss_order, _p(V))
    return V


def V_entries(xyz, tri, rows, cols, far_order=0, ss_order=5) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, float)
    tri = np.ascontiguousarray(tri, np.int32)
    rows = np.ascontiguousarray(rows, np.int64)
    cols = np.ascontiguousarray(cols, np.int64)
    out = np.empty(rows.shape[0], dtype=np.float64)
    lib().orc_V_entries(rows.shape[0], _p(rows), _p(cols), _p(xyz), _p(tri), far_order, ss_order,
                        _p(out))
    return out
