"""Pins of the CPU restatement of a frame's brick requests (tests/footprint_cpu.py).

The restatement is what the GPU footprint is compared with, so it is pinned first against things fixed
independently of it: the bricks a straight ray passes (every brick whose box the ray crosses, ordered by
entry, found here by clipping the ray against each brick box in float64), closed-form cases (a ray down
the z axis through a column of bricks, empty-space skipping, the stop at an opaque root), and the LOD
rule t = clamp(floor(log2(d / f_px)), 0, N) evaluated in float64 away from its thresholds.
"""
import math

import numpy as np

from tests import footprint_cpu as F


def _cam(pos, fwd, up=(0.0, 0.0, 1.0), f_px=100.0, w=1, h=1):
    fwd = np.asarray(fwd, np.float64)
    fwd = fwd / np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    return {"pos": np.asarray(pos, np.float32), "right": right.astype(np.float32), "up": upv.astype(np.float32),
            "fwd": fwd.astype(np.float32), "f_px": np.float32(f_px), "width": w, "height": h}


def test_ray_down_a_column_requests_every_non_empty_brick_until_an_opaque_root():
    dims, b = (64, 64, 128), 16  # grid 4 x 4 x 8
    G = (4, 4, 8)
    # camera above the volume, looking down -z through voxel (40, 24): column (2, 1, *)
    cam = _cam((40.0, 24.0, 300.0), (0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0))
    flags = np.ones(4 * 4 * 8, np.uint8)  # every brick holds an opaque label, no opaque root
    col = [2 + G[0] * (1 + G[1] * z) for z in range(8)]
    got = F.frame(cam, dims, b, flags, max_nonempty=0)
    assert [k for k, _ in got] == sorted(col)
    # bricks z = 7, 6 empty (skipped), z = 3 has an opaque root: requests z = 5, 4, 3 only
    flags[col[7]] = flags[col[6]] = 0
    flags[col[3]] = 3
    assert [k for k, _ in F.frame(cam, dims, b, flags, max_nonempty=0)] == sorted(col[3:6])
    # max_nonempty = 2: z = 5, 4
    assert [k for k, _ in F.frame(cam, dims, b, flags, max_nonempty=2)] == sorted(col[4:6])
    # the walk itself is the whole column, top down
    assert F.walk(cam, dims, b, 0, 0) == [(2, 1, z) for z in range(7, -1, -1)]


def test_lod_rule_closed_form():
    # brick (0, 0, 0) of b = 32, centre (16, 16, 16); camera on the x axis at distance d from the centre
    b, N, f_px = 32, 5, 100.0
    for d, want in ((50.0, 0), (150.0, 0), (250.0, 1), (390.0, 1), (410.0, 2), (900.0, 3), (1700.0, 4),
                    (3300.0, 5), (10 ** 6, 5)):
        cam = _cam((16.0 + d, 16.0, 16.0), (-1.0, 0.0, 0.0), f_px=f_px)
        assert F.lod_of(cam, b, N, (0, 0, 0)) == want == min(N, max(0, math.floor(math.log2(d / f_px))))


def _brick_intervals(o, d, dims, b):
    """float64: every brick whose box the ray o + t d (t >= 0, inside the volume box) crosses, by entry."""
    G = [-(-int(x) // b) for x in dims]
    out = []
    for bz in range(G[2]):
        for by in range(G[1]):
            for bx in range(G[0]):
                lo = np.array([bx, by, bz], np.float64) * b
                hi = np.minimum(lo + b, np.asarray(dims, np.float64))
                t0, t1 = 0.0, np.inf
                for a in range(3):
                    if d[a] == 0:
                        if not (lo[a] <= o[a] <= hi[a]):
                            t0, t1 = 1.0, 0.0
                        continue
                    u0, u1 = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
                    t0, t1 = max(t0, min(u0, u1)), min(t1, max(u0, u1))
                if t1 > t0:
                    out.append((t0, t1, (bx, by, bz)))
    out.sort()
    return out


def test_walk_equals_brick_box_clipping_on_random_rays():
    rng = np.random.default_rng(12)
    dims, b = (96, 64, 80), 16
    checked = 0
    for trial in range(60):
        inside = trial % 3 == 0
        pos = rng.uniform(5, 59, 3) if inside else rng.uniform(-150, 250, 3)
        target = rng.uniform(0, 64, 3) * np.array([1.5, 1.0, 1.25])
        cam = _cam(pos, target - pos, f_px=float(rng.uniform(20, 80)), w=7, h=5)
        for y in range(cam["height"]):
            for x in range(cam["width"]):
                f = lambda v: np.float64(np.float32(v))
                px = (f(x) + 0.5 - 0.5 * cam["width"]) / f(cam["f_px"])
                py = (f(y) + 0.5 - 0.5 * cam["height"]) / f(cam["f_px"])
                d = np.array([f(cam["fwd"][a]) + px * f(cam["right"][a]) - py * f(cam["up"][a]) for a in range(3)])
                o = np.array([f(v) for v in cam["pos"]])
                ref = _brick_intervals(o, d, dims, b)
                # skip grazing rays: a brick crossed over a tiny stretch, or two entries almost tied
                span = np.linalg.norm(d)
                if any((t1 - t0) * span < 1e-2 for t0, t1, _ in ref) or \
                        any((ref[i + 1][0] - ref[i][0]) * span < 1e-2 for i in range(len(ref) - 1)):
                    continue
                got = F.walk(cam, dims, b, x, y)
                assert (got or []) == [k for _, _, k in ref], (trial, x, y)
                checked += 1
    assert checked > 800
