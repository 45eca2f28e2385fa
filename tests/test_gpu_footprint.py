"""The footprint kernel (csgv_footprint_*): the brick requests of rendered frames, against the CPU
restatement in tests/footprint_cpu.py (itself pinned in tests/test_footprint_cpu.py).

Requests are integer decisions taken from IEEE single-precision arithmetic in the same operation order
on both sides, so the lists must be equal (tolerance zero).  The volume has empty bricks (skipped) and
bricks whose root label is opaque (rays stop there); cameras outside and inside the volume; several
frames of one footprint in a row (the per-brick integers are reset between frames).
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests import footprint_cpu as F

pytestmark = pytest.mark.gpu


def _flags(vol, b):
    N = b.bit_length() - 1
    Z, Y, X = vol.shape
    gx, gy, gz = -(-X // b), -(-Y // b), -(-Z // b)
    roots = []
    for k in range(gx * gy * gz):
        bx, by, bz = k % gx, (k // gx) % gy, k // (gx * gy)
        zz = np.minimum(np.arange(bz * b, bz * b + b), Z - 1)
        yy = np.minimum(np.arange(by * b, by * b + b), Y - 1)
        xx = np.minimum(np.arange(bx * b, bx * b + b), X - 1)
        roots.append(int(O.pyramid(vol[np.ix_(zz, yy, xx)])[N][0][0, 0, 0]))
    return F.brick_flags(vol, b, roots)


@pytest.mark.parametrize("b,max_nonempty", [(8, 1), (8, 0), (16, 2)])
def test_footprint_equals_cpu_restatement(b, max_nonempty):
    import torch
    import paper_2308_16619_b300 as csgv
    shape = (80, 48, 64)  # z, y, x
    vol = synth.voronoi(shape, 60, seed=3, warp_amp=2, bg_permille=500)
    Z, Y, X = shape
    dims = (X, Y, Z)
    flags = _flags(vol, b)
    assert (flags & 1 == 0).any() and (flags & 2).any() and ((flags & 3) == 1).any()
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    v = csgv.csgv_encode_bricks(d, b, csgv.csgv_build_freq_table(d, b, 1))
    fp = csgv.Footprint(v, max_nonempty=max_nonempty)
    cams = synth.camera_path(dims, 5, seed=7, width=48, height=36, fov_deg=50.0)
    inside = dict(cams[0])
    inside["pos"] = np.array([30.5, 20.25, 41.0], np.float32)
    cams.append(inside)
    n_frames_with_requests = 0
    for cam in cams:
        want = F.frame(cam, dims, b, flags, max_nonempty)
        bricks, lods = fp.frame(csgv.make_camera(cam["pos"], cam["right"], cam["up"], cam["fwd"], cam["f_px"],
                                                 cam["width"], cam["height"]))
        got = list(zip(bricks.cpu().numpy().tolist(), lods.cpu().numpy().tolist()))
        assert got == want
        n_frames_with_requests += len(want) > 0
    assert n_frames_with_requests >= 5
    fp.close()
    v.close()
