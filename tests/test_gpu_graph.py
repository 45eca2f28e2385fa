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
    assert best.rans_ctas_per_sm in (4, 5) and 0 < best.ms < 1e3
    out.fill_(-1)
    csgv.csgv_decode_bricks(v, t["ids"], t["lods"], out, t["offs"], st)
    torch.cuda.synchronize()
    assert bool((st == 0).all()) and torch.equal(out, ref)
