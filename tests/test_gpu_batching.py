"""Batched decoding at scale: the 1024^3 packed-ellipsoid volume, 60 000 requests over all 32 768
bricks of 32^3 at random LOD 0..5 (uneven stream lengths, duplicates), decoded in one persistent launch.

Checked against the oracle on a seeded sample of requests (the oracle's pyramid of the same brick),
plus the invariant that every request decodes alone to the same bytes as inside the batch.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

_cache = {}


def cells_volume():
    if "vol" not in _cache:
        _cache["vol"] = synth.make("cells1024")
    return _cache["vol"]


def batch_requests(n_bricks, n=60000, seed=3):
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, n_bricks, size=n).astype(np.uint32)
    lods = rng.integers(0, 6, size=n).astype(np.uint8)
    return ids, lods


def brick_of(vol, b, bid):
    Z, Y, X = vol.shape
    nbx, nby = X // b, Y // b
    bx, by, bz = bid % nbx, (bid // nbx) % nby, bid // (nbx * nby)
    return np.ascontiguousarray(vol[bz * b:(bz + 1) * b, by * b:(by + 1) * b, bx * b:(bx + 1) * b])


def test_cells1024_mixed_lod_batch():
    import torch
    import paper_2308_16619_b300 as csgv
    vol = cells_volume()
    b = 32
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    table = csgv.csgv_build_freq_table(d, b, 512)
    v = csgv.csgv_encode_bricks(d, b, table)
    del d
    n_bricks = v.info().n_bricks
    assert n_bricks == 32768
    ids, lods = batch_requests(n_bricks)
    offs, total = csgv.request_layout(b, lods)
    assert abs(total * 4 / 1e9 - 1.5) < 0.05  # about 1.5 GB of labels, mean 6241.5 voxels per request
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    status = torch.full((len(ids),), -1, dtype=torch.int32, device="cuda")
    ids_d = torch.from_numpy(ids.view(np.int32)).cuda()
    lods_d = torch.from_numpy(lods).cuda()
    offs_d = torch.from_numpy(offs).cuda()
    csgv.csgv_decode_bricks(v, ids_d, lods_d, out, offs_d, status)
    torch.cuda.synchronize()
    assert bool((status == 0).all())
    rng = np.random.default_rng(11)
    sample = rng.choice(len(ids), size=400, replace=False)
    out_h = out.cpu().numpy().view(np.uint32)
    for r in sample:
        t = int(lods[r])
        B = b >> t
        got = out_h[offs[r]:offs[r] + B ** 3].reshape(B, B, B)
        want = O.pyramid(brick_of(vol, b, int(ids[r])))[t][0]
        assert np.array_equal(got, want), (r, int(ids[r]), t)
    # each request alone gives the same bytes as inside the batch
    for r in sample[:40]:
        t = int(lods[r])
        B3 = (b >> t) ** 3
        o1 = torch.empty(B3, dtype=torch.int32, device="cuda")
        s1 = torch.empty(1, dtype=torch.int32, device="cuda")
        z = torch.zeros(1, dtype=torch.int64, device="cuda")
        csgv.csgv_decode_bricks(v, ids_d[r:r + 1], lods_d[r:r + 1], o1, z, s1)
        torch.cuda.synchronize()
        assert int(s1.item()) == 0
        assert np.array_equal(o1.cpu().numpy().view(np.uint32), out_h[offs[r]:offs[r] + B3])
    v.close()


def test_large_mixed_batch_split_by_lod_equals_oracle_and_small_batches():
    """A batch of 32^3 requests large enough that the rebuild runs the LOD 0..1 requests and the LOD >= 2
    requests in separate kernels (one CTA size each) gives the oracle's labels and the same bytes as the
    same requests decoded in batches too small for that split."""
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((128, 128, 128), 150, seed=21, warp_amp=3, bg_permille=300)
    V = O.encode_volume(vol, 5, stride=1)
    gv = csgv.csgv_volume_import(5, V.dims, V.K_max, V.S_min, V.freq, V.pal_off, V.pal, V.int_off, V.int_words,
                                 V.leaf_off, V.leaf_words, V.n_int_sym, V.n_leaf_sym)
    rng = np.random.default_rng(22)
    n = 9000
    ids = rng.integers(0, V.n_bricks, size=n).astype(np.uint32)
    lods = rng.integers(0, 6, size=n).astype(np.uint8)
    offs, total = csgv.request_layout(32, lods)
    ids_d = torch.from_numpy(ids.view(np.int32)).cuda()
    lods_d = torch.from_numpy(lods).cuda()
    offs_d = torch.from_numpy(np.asarray(offs, np.int64)).cuda()
    out = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((n,), -99, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(gv, ids_d, lods_d, out, offs_d, status)
    ref, roff, rst = O.decode_bricks(V, ids, lods)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all() and (rst == 0).all()
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)
    out2 = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    status2 = torch.full((n,), -99, dtype=torch.int32, device="cuda")
    for r0 in range(0, n, 2000):
        r1 = min(n, r0 + 2000)
        csgv.csgv_decode_bricks(gv, ids_d[r0:r1], lods_d[r0:r1], out2, offs_d[r0:r1], status2[r0:r1])
    torch.cuda.synchronize()
    assert (status2.cpu().numpy() == 0).all()
    assert np.array_equal(out2.cpu().numpy().view(np.uint32), got)


@pytest.mark.parametrize("mix", ["all_lod1", "coarse_and_few_fine", "all_lod0"])
def test_large_batch_split_with_empty_classes(mix):
    """Large batches whose LOD classes are lopsided or empty (the per-class rebuild kernels find nothing to
    do, or all of it) give the oracle's labels and statuses."""
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((128, 128, 128), 120, seed=23, warp_amp=2, bg_permille=200)
    V = O.encode_volume(vol, 5, stride=1)
    gv = csgv.csgv_volume_import(5, V.dims, V.K_max, V.S_min, V.freq, V.pal_off, V.pal, V.int_off, V.int_words,
                                 V.leaf_off, V.leaf_words, V.n_int_sym, V.n_leaf_sym)
    rng = np.random.default_rng(24)
    n = 8500
    ids = rng.integers(0, V.n_bricks, size=n).astype(np.uint32)
    if mix == "all_lod1":
        lods = np.ones(n, np.uint8)
    elif mix == "all_lod0":
        lods = np.zeros(n, np.uint8)
    else:
        lods = rng.integers(2, 6, size=n).astype(np.uint8)
        lods[rng.choice(n, size=5, replace=False)] = 0
    offs, total = csgv.request_layout(32, lods)
    out = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((n,), -99, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(gv, torch.from_numpy(ids.view(np.int32)).cuda(), torch.from_numpy(lods).cuda(), out,
                            torch.from_numpy(np.asarray(offs, np.int64)).cuda(), status)
    ref, _, rst = O.decode_bricks(V, ids, lods)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all() and (rst == 0).all()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)


def test_empty_batch_is_a_no_op():
    """No requests: the decode, the plain decode and the autotuner return at once, write nothing and leave
    the volume's launch shape as it was."""
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((64, 64, 64), 30, seed=25, warp_amp=2, bg_permille=200)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    v = csgv.csgv_encode_bricks(d, 32, csgv.csgv_build_freq_table(d, 32, 1))
    before = csgv.csgv_decode_get_tuning(v).as_dict()
    ids = torch.empty(0, dtype=torch.int32, device="cuda")
    lods = torch.empty(0, dtype=torch.uint8, device="cuda")
    offs = torch.empty(0, dtype=torch.int64, device="cuda")
    st = torch.empty(0, dtype=torch.int32, device="cuda")
    out = torch.full((16,), -7, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(v, ids, lods, out, offs, st)
    csgv.csgv_decode_bricks_plain(v, ids, lods, out, offs, st)
    best = csgv.csgv_decode_autotune(v, ids, lods, out, offs, st)
    torch.cuda.synchronize()
    assert bool((out == -7).all())
    assert csgv.csgv_decode_get_tuning(v).as_dict() == before
    assert dict(best.as_dict(), ms=0.0) == dict(before, ms=0.0)
    v.close()
