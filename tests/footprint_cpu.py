"""Plain CPU restatement of a frame's brick requests (csgv_footprint_frame), for the tests.

What it computes (Sec. 4 of the paper, "Raymarching" and "Empty-Space Skipping", with the readings
stated in include/csgv.h): one ray per pixel through the pixel centre, clipped to the volume box
[0, dims), walks the brick grid one brick at a time; a brick with no opaque label (label 0 is the
only transparent one) is skipped, any other is requested at LOD clamp(floor(log2(d / f_px)), 0, N),
d the distance from the camera to the brick centre; the ray stops at a brick whose root label is
opaque, or once it has requested max_nonempty bricks (0: no limit).

Floating point: every operation is one IEEE single-precision operation on numpy float32 scalars,
in the order the CUDA kernel takes them (that kernel uses explicitly rounded operations and no fused
multiply-adds), so both take the same integer decisions (which brick comes next, which LOD).  The
restatement shares no code with the library.
"""
import numpy as np

f32 = np.float32
PARALLEL = f32(1e-30)


def brick_flags(vol, b, root_labels):
    """bit 0: the brick holds a non-zero label; bit 1: its root label (mode of the whole brick) is
    non-zero.  vol is [Z, Y, X]; bricks padded by clamp-to-edge; root_labels[k] given by the caller."""
    Z, Y, X = vol.shape
    gx, gy, gz = -(-X // b), -(-Y // b), -(-Z // b)
    flags = np.zeros(gx * gy * gz, np.uint8)
    for k in range(len(flags)):
        bx, by, bz = k % gx, (k // gx) % gy, k // (gx * gy)
        zz = np.minimum(np.arange(bz * b, bz * b + b), Z - 1)
        yy = np.minimum(np.arange(by * b, by * b + b), Y - 1)
        xx = np.minimum(np.arange(bx * b, bx * b + b), X - 1)
        any_opaque = bool((vol[np.ix_(zz, yy, xx)] != 0).any())
        flags[k] = (1 if any_opaque else 0) | (2 if root_labels[k] != 0 else 0)
    return flags


def _walk(cam, dims, b, px_i, py_i):
    """The bricks one ray passes, in order, as (bx, by, bz) and the ray parameter bound; None if it misses."""
    o = [f32(v) for v in cam["pos"]]
    right = [f32(v) for v in cam["right"]]
    up = [f32(v) for v in cam["up"]]
    fwd = [f32(v) for v in cam["fwd"]]
    f_px = f32(cam["f_px"])
    half_w, half_h = f32(0.5) * f32(cam["width"]), f32(0.5) * f32(cam["height"])
    D = [f32(d) for d in dims]
    B = f32(b)
    G = [-(-int(d) // b) for d in dims]
    px = (f32(px_i) + f32(0.5) - half_w) / f_px
    py = (f32(py_i) + f32(0.5) - half_h) / f_px
    d, inv = [f32(0)] * 3, [f32(0)] * 3
    tn, tf = f32(-np.inf), f32(np.inf)
    for a in range(3):
        d[a] = (fwd[a] + px * right[a]) - py * up[a]
        if abs(d[a]) < PARALLEL:
            d[a] = f32(0)
            if o[a] < f32(0) or o[a] > D[a]:
                return None
            continue
        inv[a] = f32(1) / d[a]
        t0 = (f32(0) - o[a]) * inv[a]
        t1 = (D[a] - o[a]) * inv[a]
        tn = max(tn, min(t0, t1))
        tf = min(tf, max(t0, t1))
    t = max(tn, f32(0))
    if not (tf >= t) or not (tf > f32(0)):
        return None
    idx, step, tmax, tdel = [0] * 3, [0] * 3, [f32(0)] * 3, [f32(0)] * 3
    for a in range(3):
        p = o[a] + d[a] * t
        i = int(np.floor(p / B))
        idx[a] = min(max(i, 0), G[a] - 1)
        step[a] = 1 if d[a] > 0 else (-1 if d[a] < 0 else 0)
        if step[a] == 0:
            tmax[a], tdel[a] = f32(np.inf), f32(np.inf)
        else:
            bound = f32((idx[a] + (1 if step[a] > 0 else 0)) * b)
            tmax[a] = (bound - o[a]) * inv[a]
            tdel[a] = B * abs(inv[a])
    out = []
    for _ in range(G[0] + G[1] + G[2] + 3):
        out.append(tuple(idx))
        a = 0
        if tmax[1] < tmax[a]:
            a = 1
        if tmax[2] < tmax[a]:
            a = 2
        if tmax[a] > tf:
            break
        idx[a] += step[a]
        if idx[a] < 0 or idx[a] >= G[a]:
            break
        tmax[a] = tmax[a] + tdel[a]
    return out


def lod_of(cam, b, N, brick_xyz):
    o = [f32(v) for v in cam["pos"]]
    B = f32(b)
    d2 = f32(0)
    for a in range(3):
        c = (f32(brick_xyz[a]) + f32(0.5)) * B
        e = c - o[a]
        d2 = d2 + e * e
    thr, lv = f32(cam["f_px"]), 0
    for _ in range(N):
        thr = thr * f32(2)
        lv += 1 if d2 >= thr * thr else 0
    return lv


def frame(cam, dims, b, flags, max_nonempty=1):
    """Requests of one frame: sorted list of (brick id, LOD)."""
    N = b.bit_length() - 1
    G = [-(-int(d) // b) for d in dims]
    req = {}
    with np.errstate(over="ignore", divide="ignore", invalid="ignore"):
        for y in range(cam["height"]):
            for x in range(cam["width"]):
                bricks = _walk(cam, dims, b, x, y)
                if bricks is None:
                    continue
                hits = 0
                for bx, by, bz in bricks:
                    k = bx + G[0] * (by + G[1] * bz)
                    fl = int(flags[k])
                    if not (fl & 1):
                        continue
                    lv = lod_of(cam, b, N, (bx, by, bz))
                    assert req.get(k, lv) == lv
                    req[k] = lv
                    hits += 1
                    if (fl & 2) or (max_nonempty and hits >= max_nonempty):
                        break
    return sorted(req.items())


def walk(cam, dims, b, x, y):
    """The bricks the ray of pixel (x, y) passes, in order (for the tests)."""
    with np.errstate(over="ignore", divide="ignore", invalid="ignore"):
        return _walk(cam, dims, b, x, y)
