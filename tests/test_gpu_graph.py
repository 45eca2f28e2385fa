"""Batching at scale: a batched decode captured into a CUDA graph, and the decode autotuner.

csgv_decode_bricks issues only stream-ordered work (pool allocation, memset, kernels, free), so a batch can
be captured once and replayed; every replay must give the same bytes as a direct call.  The autotuner may
pick any configuration, but decoding afterwards must still be exact.  Integer data: the tolerance is zero.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((128, 128, 192), 300, seed=23, warp_amp=4, bg_permille=300)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    v = csgv.csgv_encode_bricks(d, 32, csgv.csgv_build_freq_table(d, 32, 1))
    rng = np.random.default_rng(9)
    n = 3000
    ids_h = rng.integers(0, v.info().n_bricks, size=n).astype(np.uint32)
    lods_h = rng.integers(0, 6, size=n).astype(np.uint8)
    offs_h, total = csgv.request_layout(32, lods_h)
    t = dict(ids=torch.from_numpy(ids_h.view(np.int32)).cuda(), lods=torch.from_numpy(lods_h).cuda(),
             offs=torch.from_numpy(offs_h).cuda(), total=total)
    ref = torch.empty(total, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(v, t["ids"], t["lods"], ref, t["offs"], st)
    torch.cuda.synchronize()
    assert bool((st == 0).all())
    yield v, t, ref
    v.close()


def test_decode_captured_in_cuda_graph_replays_bit_exact(batch):
    import torch
    import paper_2308_16619_b300 as csgv
    v, t, ref = batch
    out = torch.empty(t["total"], dtype=torch.int32, device="cuda")
    st = torch.empty(t["ids"].numel(), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up on the capture stream (pool and kernel attributes)
        csgv.csgv_decode_bricks(v, t["ids"], t["lods"], out, t["offs"], st)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        csgv.csgv_decode_bricks(v, t["ids"], t["lods"], out, t["offs"], st)
    for _ in range(3):
        out.fill_(-1)
        st.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert bool((st == 0).all())
        assert torch.equal(out, ref)


def test_autotune_keeps_decoding_exact(batch):
    import torch
    import paper_2308_16619_b300 as csgv
    v, t, ref = batch
    out = torch.empty(t["total"], dtype=torch.int32, device="cuda")
    st = torch.empty(t["ids"].numel(), dtype=torch.int32, device="cuda")
    best = csgv.csgv_decode_autotune(v, t["ids"], t["lods"], out, t["offs"], st)
    assert best.workspace_bytes in (64 << 20, 192 << 20, 512 << 20, 1024 << 20)
    assert best.rans_ctas_per_sm in (4, 5, 6) and best.ring_words in (128, 256, 512)
    assert best.rebuild_threads in (128, 256) and best.medium_threads in (64, 128, 256) and 0 < best.ms < 1e3
    assert best.compact_nodes in (0, 256, 512, 1024, 1280)
    assert csgv.csgv_decode_get_tuning(v).as_dict() == dict(best.as_dict(), ms=0.0)  # kept in the volume
    out.fill_(-1)
    csgv.csgv_decode_bricks(v, t["ids"], t["lods"], out, t["offs"], st)
    torch.cuda.synchronize()
    assert bool((st == 0).all()) and torch.equal(out, ref)


def test_every_decode_tuning_point_decodes_exactly():
    # Every launch shape the autotuner can pick (rANS ring depth x CTAs per SM, threads per LOD 0 and per LOD 1
    # request, workspace per slice; the compact/full split of LOD 0 requests cycled through its five values) on a
    # 9000-request mixed-LOD batch, which is above the size from which LOD 1
    # requests go to their own kernel; each result equals the oracle's pyramid level of every request's brick.
    import itertools
    import torch
    import oracle as O
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((128, 128, 192), 300, seed=29, warp_amp=4, bg_permille=300)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    v = csgv.csgv_encode_bricks(d, 32, csgv.csgv_build_freq_table(d, 32, 1))
    n_bricks = v.info().n_bricks
    rng = np.random.default_rng(31)
    n = 9000
    ids_h = rng.integers(0, n_bricks, size=n).astype(np.uint32)
    lods_h = rng.integers(0, 6, size=n).astype(np.uint8)
    offs_h, total = csgv.request_layout(32, lods_h)
    Z, Y, X = vol.shape
    nbx, nby = X // 32, Y // 32
    pyr = []
    for bid in range(n_bricks):
        bx, by, bz = bid % nbx, (bid // nbx) % nby, bid // (nbx * nby)
        pyr.append(O.pyramid(np.ascontiguousarray(vol[32 * bz:32 * bz + 32, 32 * by:32 * by + 32, 32 * bx:32 * bx + 32])))
    want = np.empty(total, np.uint32)
    for r in range(n):
        lv = pyr[ids_h[r]][lods_h[r]][0].ravel()
        want[offs_h[r]:offs_h[r] + lv.size] = lv
    want_d = torch.from_numpy(want.view(np.int32)).cuda()
    ids = torch.from_numpy(ids_h.view(np.int32)).cuda()
    lods = torch.from_numpy(lods_h).cuda()
    offs = torch.from_numpy(offs_h).cuda()
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    points = 0
    for ring, ctas, lt, mt, ws in itertools.product((128, 256, 512), (4, 5, 6), (128, 256), (64, 128, 256),
                                                    (64, 1024)):
        cn = (0, 256, 512, 1024, 1280)[points % 5]  # the compact/full split, cycled over the points
        tu = csgv.DecodeTuning(workspace_bytes=ws << 20, rans_ctas_per_sm=ctas, ring_words=ring, rebuild_threads=lt,
                               medium_threads=mt, compact_nodes=cn)
        if ring == 512 and ctas == 6:  # 6 x 40 KB of shared memory: refused
            with pytest.raises(csgv.CsgvError):
                csgv.csgv_decode_set_tuning(v, tu)
            continue
        csgv.csgv_decode_set_tuning(v, tu)
        out.fill_(-1)
        st.fill_(-1)
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, st)
        torch.cuda.synchronize()
        assert bool((st == 0).all()), tu.as_dict()
        assert torch.equal(out, want_d), tu.as_dict()
        points += 1
    assert points == 8 * 2 * 3 * 2
    v.close()
