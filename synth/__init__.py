"""Seeded synthetic label volumes standing in for the paper's data sets.

This module holds no codec arithmetic; it only makes uint32 label volumes
(numpy arrays shaped [Z, Y, X], x fastest) that the CPU oracle and the CUDA
library both consume.  Recipes (sizes, seeds, structure) are listed in
WORKLOADS and documented beside each generator in gen.c.
"""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gen.c")
LIB = os.path.join(HERE, "libsynth.so")

_lib = None


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC", "-pthread", SRC, "-o", tmp,
                           "-lm"])
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.synth_voronoi.restype = C.c_int
        _lib.synth_voronoi.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint64,
                                       C.c_int, C.c_uint32, C.c_int]
        _lib.synth_ellipsoids.restype = C.c_uint64
        _lib.synth_ellipsoids.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64,
                                          C.c_double, C.c_double, C.c_double, C.c_uint64]
        _lib.synth_label.restype = C.c_uint32
        _lib.synth_label.argtypes = [C.c_uint64, C.c_uint64]
    return _lib


def _threads(n):
    return n or max(1, os.cpu_count() or 1)


def voronoi(shape_zyx, n_sites, seed, warp_amp=0, bg_permille=0, n_threads=None, out=None):
    Z, Y, X = shape_zyx
    vol = out if out is not None else np.empty((Z, Y, X), np.uint32)
    rc = lib().synth_voronoi(vol.ctypes.data_as(C.c_void_p), X, Y, Z, n_sites, seed, warp_amp, bg_permille,
                             _threads(n_threads))
    assert rc == 0
    return vol


def ellipsoids(shape_zyx, n_target, seed, len_lo=12.0, len_hi=40.0, short_lo=4.0, max_attempts=None):
    Z, Y, X = shape_zyx
    vol = np.zeros((Z, Y, X), np.uint32)
    placed = lib().synth_ellipsoids(vol.ctypes.data_as(C.c_void_p), X, Y, Z, n_target, seed, len_lo, len_hi,
                                    short_lo, max_attempts or 20 * n_target)
    return vol, int(placed)


# Workload recipes.  "small" is the 128^3 plain-method case; "voronoi512" the
# 512^3 warped Voronoi with 30 % background; "cells1024" the 1024^3 packed
# ellipsoid cells used for mixed-LOD batching.
WORKLOADS = {
    "voronoi128": dict(shape=(128, 128, 128), make=lambda: voronoi((128, 128, 128), 150, seed=1)),
    "voronoi512": dict(shape=(512, 512, 512),
                       make=lambda: voronoi((512, 512, 512), 20000, seed=2, warp_amp=4, bg_permille=300)),
    "cells1024": dict(shape=(1024, 1024, 1024), make=lambda: ellipsoids((1024, 1024, 1024), 200000, seed=3)[0]),
}


def make(name):
    return WORKLOADS[name]["make"]()
