"""Detail separation (Sec. 4.2): the leaf streams live in mapped host memory and decoding reads them in
place.  Every LOD must decode to the oracle's labels and to the same bytes as with all data on the device
(integer data, tolerance zero), coarse LODs must not need the leaf data, and moving the leaves back must
restore the volume."""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def decode_all(csgv, torch, v, ids, lods, offs, total):
    out = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    st = torch.full((ids.numel(),), -1, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(v, ids, lods, out, offs, st)
    torch.cuda.synchronize()
    assert bool((st == 0).all())
    return out.cpu().numpy()


def test_leaves_in_host_memory_decode_every_lod_exactly():
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((128, 128, 128), 500, seed=41, warp_amp=4, bg_permille=300)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    v = csgv.csgv_encode_bricks(d, 32, csgv.csgv_build_freq_table(d, 32, 1))
    n = v.info().n_bricks
    rng = np.random.default_rng(4)
    ids_h = rng.integers(0, n, size=500).astype(np.uint32)
    lods_h = rng.integers(0, 6, size=500).astype(np.uint8)
    offs_h, total = csgv.request_layout(32, lods_h)
    ids = torch.from_numpy(ids_h.view(np.int32)).cuda()
    lods = torch.from_numpy(lods_h).cuda()
    offs = torch.from_numpy(offs_h).cuda()
    ref = decode_all(csgv, torch, v, ids, lods, offs, total)
    want, want_off, st = O.decode_bricks(O.encode_volume(vol, 5, stride=1), ids_h, lods_h)
    assert (st == 0).all() and np.array_equal(want_off.astype(np.int64), offs_h)
    assert np.array_equal(ref.view(np.uint32), want[:total])
    before = v.export()
    v.leaves_to_host()
    host = decode_all(csgv, torch, v, ids, lods, offs, total)
    assert np.array_equal(host.view(np.uint32), want[:total])  # leaves read over the host link: the oracle's labels
    assert np.array_equal(host, ref)
    assert np.array_equal(v.export()["leaf_words"], before["leaf_words"])
    v.leaves_to_device()
    assert np.array_equal(decode_all(csgv, torch, v, ids, lods, offs, total), ref)
    v.close()
