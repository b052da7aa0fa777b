"""Loader for the CPU uniform-grid timing baseline (ug_cpu.cpp): compiles it
with g++ -O3 -fopenmp next to the source when missing or stale, and runs it on
float32 rows through ctypes.  Used by the benchmark; it is not the library and
not the test oracle."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ug_cpu.cpp")
LIB = os.path.join(HERE, "libugcpu.so")


class _Params(ctypes.Structure):
    _fields_ = [(f, ctypes.c_float) for f in
                ("k", "gamma", "adherence", "dt", "density", "max_disp", "contact_margin")]


def build() -> str:
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["g++", "-O3", "-fopenmp", "-std=c++17", "-shared", "-fPIC", SRC, "-o", LIB],
                       check=True)
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.ugcpu_steps.restype = ctypes.c_double
        _lib.ugcpu_steps.argtypes = [ctypes.c_void_p, ctypes.c_uint32, _Params, ctypes.c_int,
                                     ctypes.c_int]
        _lib.ugcpu_max_threads.restype = ctypes.c_int
    return _lib


def max_threads() -> int:
    return int(load().ugcpu_max_threads())


def steps(rows: np.ndarray, nsteps: int = 1, threads: int = 0, k=2.0, gamma=1.0, adherence=0.1,
          dt=1.0, density=0.02, max_disp=3.0, contact_margin=0.0):
    """Advance a copy of `rows` ((n, 4) float32) by nsteps; returns (rows, seconds)."""
    lib = load()
    r = np.ascontiguousarray(rows, dtype=np.float32).copy()
    p = _Params(k, gamma, adherence, dt, density, max_disp, contact_margin)
    secs = lib.ugcpu_steps(r.ctypes.data, len(r), p, int(nsteps), int(threads))
    return r, float(secs)
