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
GPU_SRC = os.path.join(HERE, "gen_gpu.cu")
GPU_LIB = os.path.join(HERE, "libsynth_gpu.so")

_lib = None
_gpu_lib = None


def build_gpu(force=False):
    if not force and os.path.exists(GPU_LIB) and os.path.getmtime(GPU_LIB) >= os.path.getmtime(GPU_SRC):
        return GPU_LIB
    tmp = GPU_LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-shared", "-Xcompiler", "-fPIC", GPU_SRC, "-o", tmp])
    os.replace(tmp, GPU_LIB)
    return GPU_LIB


def gpu_lib():
    global _gpu_lib
    if _gpu_lib is None:
        _gpu_lib = C.CDLL(build_gpu())
        _gpu_lib.synth_worley_dev.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32,
                                              C.c_uint64, C.c_void_p]
        _gpu_lib.synth_fiber_bricks_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint32, C.c_uint64,
                                                    C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                                    C.c_uint64, C.c_void_p]
    return _gpu_lib


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
        _lib.synth_worley.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint64,
                                      C.c_int]
        _lib.synth_fibers.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                      C.c_uint64]
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


def worley(shape_zyx, cell, seed, n_threads=None):
    """Worley F1 cells on a jittered grid (host): label = hash of the nearest of the 27 neighbouring features."""
    Z, Y, X = shape_zyx
    vol = np.empty((Z, Y, X), np.uint32)
    assert lib().synth_worley(vol.ctypes.data_as(C.c_void_p), X, Y, Z, cell, seed, _threads(n_threads)) == 0
    return vol


def worley_device(shape_zyx, cell, seed):
    """Same volume made on the current CUDA device; returns an int32-typed torch tensor of the uint32 labels."""
    import torch
    Z, Y, X = shape_zyx
    vol = torch.empty((Z, Y, X), dtype=torch.int32, device="cuda")
    rc = gpu_lib().synth_worley_dev(C.c_void_p(vol.data_ptr()), X, Y, Z, cell, seed,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    return vol


def fibers(shape_zyx, cell, tubes, seed):
    """Fiber volume (host, small volumes): tubes along Catmull-Rom splines, `tubes` per cell of cell^3 voxels
    (gen.c, synth_fibers)."""
    Z, Y, X = shape_zyx
    vol = np.empty((Z, Y, X), np.uint32)
    assert lib().synth_fibers(vol.ctypes.data_as(C.c_void_p), X, Y, Z, cell, tubes, seed) == 0
    return vol


def fiber_bricks_device(dims_xyz, b, cell, tubes, seed, first=0, m=None, ids=None, out=None):
    """Bricks of the same fiber volume made on the current CUDA device without the volume: brick ids
    first .. first + m - 1 (or the int64 device tensor `ids`), each b^3 labels x fastest, brick-major, in an
    int32-typed torch tensor (out, if given)."""
    import torch
    X, Y, Z = dims_xyz
    if ids is not None:
        m = ids.numel()
    if out is None:
        out = torch.empty(m * b ** 3, dtype=torch.int32, device="cuda")
    rc = gpu_lib().synth_fiber_bricks_dev(C.c_void_p(out.data_ptr()),
                                          C.c_void_p(ids.data_ptr() if ids is not None else 0), first, m, X, Y, Z,
                                          b, cell, tubes, seed, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    return out


def camera_path(dims_xyz, n_frames, seed, width=1920, height=1080, fov_deg=45.0, r_lo=1.05, r_hi=1.9):
    """Cameras of a fly-around, one per frame: dicts of float32 pos / right / up / fwd (voxel units),
    f_px (focal length in pixels), width and height.

    The camera follows a closed uniform Catmull-Rom spline through 8 seeded points on a shell around the
    volume (radius r_lo..r_hi times the half diagonal) and looks at the centre, z up; vertical field of
    view fov_deg.  The brick requests of each frame come from the library's footprint kernel."""
    X, Y, Z = dims_xyz
    size = np.array([X, Y, Z], np.float64)
    centre = size / 2
    half_diag = float(np.linalg.norm(size / 2))
    rng = np.random.default_rng(seed)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radii = rng.uniform(r_lo, r_hi, size=8) * half_diag
    ctrl = dirs * radii[:, None] + centre
    f_px = (height / 2) / np.tan(np.radians(fov_deg) / 2)
    cams = []
    for f in range(n_frames):
        u = 8.0 * f / n_frames
        k = int(u)
        t = u - k
        p0, p1, p2, p3 = (ctrl[(k + d) % 8] for d in (-1, 0, 1, 2))
        cam = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t * t +
                     (-p0 + 3 * p1 - 3 * p2 + p3) * t * t * t)
        fwd = centre - cam
        fwd /= np.linalg.norm(fwd)
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        cams.append({"pos": cam.astype(np.float32), "right": right.astype(np.float32), "up": up.astype(np.float32),
                     "fwd": fwd.astype(np.float32), "f_px": np.float32(f_px), "width": int(width),
                     "height": int(height)})
    return cams


# Workload recipes.  "small" is the 128^3 plain-method case; "voronoi512" the
# 512^3 warped Voronoi with 30 % background; "cells1024" the 1024^3 packed
# ellipsoid cells used for mixed-LOD batching.
WORKLOADS = {
    "voronoi128": dict(shape=(128, 128, 128), make=lambda: voronoi((128, 128, 128), 150, seed=1)),
    "voronoi512": dict(shape=(512, 512, 512),
                       make=lambda: voronoi((512, 512, 512), 20000, seed=2, warp_amp=4, bg_permille=300)),
    "cells1024": dict(shape=(1024, 1024, 1024), make=lambda: ellipsoids((1024, 1024, 1024), 200000, seed=3)[0]),
    # 4096 x 4096 x 2048 fibers: 1M tubes (8 per 64^3 cell), made brick by brick on the device, never whole
    "fiber4096": dict(shape=(2048, 4096, 4096), cell=64, tubes=8, seed=5, make=None),
    # 2048 x 2048 x 1024 Worley cells on a 24-voxel jittered grid (made on the device: 16 GB)
    "worley2048": dict(shape=(1024, 2048, 2048), make=lambda: worley_device((1024, 2048, 2048), 24, seed=4)),
}


def make(name):
    return WORKLOADS[name]["make"]()
