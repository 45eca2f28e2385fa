"""The decode server (csgv_serve_*): continuous batching over a device cache of decoded bricks.

Every served result must equal the oracle's decode of the same request and the same request decoded
alone by csgv_decode_bricks (bit-exact), whatever else was in flight; the cache must hit on repeats, evict least recently used entries when
full, and hold back requests (admission by free memory) until releases free space.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served_volume():
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((128, 192, 256), 400, seed=17, warp_amp=4, bg_permille=300)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    t = csgv.csgv_build_freq_table(d, 32, 1)
    v = csgv.csgv_encode_bricks(d, 32, t)
    v.oracle = O.encode_volume(vol, 5, stride=1)  # the CPU oracle's encoding of the same volume
    yield v
    v.close()


def decode_alone(v, brick, lod):
    import torch
    import paper_2308_16619_b300 as csgv
    B3 = (32 >> lod) ** 3
    out = torch.empty(B3, dtype=torch.int32, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(v, torch.tensor([brick], dtype=torch.int32, device="cuda"),
                            torch.tensor([lod], dtype=torch.uint8, device="cuda"), out,
                            torch.zeros(1, dtype=torch.int64, device="cuda"), st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return out.cpu().numpy().view(np.uint32)


def check_results(srv, v, bricks, lods, res):
    bricks = np.asarray(bricks, np.uint32)
    lods = np.asarray(lods, np.uint8)
    want, off, st = O.decode_bricks(v.oracle, bricks, lods)
    assert (st == 0).all()
    for k, (br, lod, r) in enumerate(zip(bricks, lods, res)):
        assert r.status == 0 and r.brick == br and r.lod == lod
        got = srv.labels(r, 32).cpu().numpy().view(np.uint32)
        B3 = (32 >> int(lod)) ** 3
        assert np.array_equal(got, want[int(off[k]):int(off[k]) + B3])
        assert np.array_equal(got, decode_alone(v, int(br), int(lod)))


def test_served_results_equal_alone_under_continuous_batching(served_volume):
    import paper_2308_16619_b300 as csgv
    v = served_volume
    n_bricks = v.info().n_bricks
    srv = csgv.Server(v, cache_bytes=1 << 30, n_streams=3)
    rng = np.random.default_rng(5)
    # many tickets submitted back to back: later ones are admitted while earlier batches run
    tickets = []
    for k in range(24):
        m = int(rng.integers(1, 200))
        bricks = rng.integers(0, n_bricks, size=m).astype(np.uint32)
        lods = rng.integers(0, 6, size=m).astype(np.uint8)
        tickets.append((srv.submit(bricks, lods), bricks, lods))
    for t, bricks, lods in tickets:
        rc, res = srv.poll(t, timeout_us=30_000_000)
        assert rc == csgv.CSGV_OK
        idx = rng.choice(len(bricks), size=min(8, len(bricks)), replace=False)
        check_results(srv, v, bricks[idx], lods[idx], [res[i] for i in idx])
        srv.release(t)
    st, lat = srv.stats(with_latencies=True)
    assert st["submitted"] == 24 and len(lat) == 24 and st["batches"] >= 2
    assert st["hits"] + st["shared"] + st["misses"] == sum(len(b) for _, b, _ in tickets)
    # repeats are cache hits and give the same bytes
    t0, bricks, lods = tickets[0]
    h0 = st["hits"]
    t = srv.submit(bricks, lods)
    rc, res = srv.poll(t, timeout_us=10_000_000)
    assert rc == csgv.CSGV_OK
    check_results(srv, v, bricks[:5], lods[:5], res[:5])
    srv.release(t)
    assert srv.stats()[0]["hits"] >= h0 + len(set(zip(bricks.tolist(), lods.tolist())))
    srv.close()


def test_eviction_admission_and_range_errors(served_volume):
    import paper_2308_16619_b300 as csgv
    v = served_volume
    n_bricks = v.info().n_bricks
    slot = 32 ** 3 * 4
    srv = csgv.Server(v, cache_bytes=12 * slot, n_streams=2)  # room for 12 bricks at LOD 0
    a = np.arange(0, 8, dtype=np.uint32)
    b_ = np.arange(8, 16, dtype=np.uint32)
    z = np.zeros(8, np.uint8)
    ta = srv.submit(a, z)
    rc, res_a = srv.poll(ta, timeout_us=10_000_000)
    assert rc == csgv.CSGV_OK
    # ticket B needs 8 more slots while A's 8 stay pinned: only 4 are free, so B waits
    tb = srv.submit(b_, z)
    rc, _ = srv.poll(tb, timeout_us=200_000)
    assert rc == csgv.CSGV_ERR_TIMEOUT
    check_results(srv, v, a[:3], z[:3], res_a[:3])
    srv.release(ta)  # A's entries become evictable: B is admitted by evicting them
    rc, res_b = srv.poll(tb, timeout_us=10_000_000)
    assert rc == csgv.CSGV_OK
    check_results(srv, v, b_, z, res_b)
    srv.release(tb)
    st, _ = srv.stats()
    assert st["evictions"] >= 4
    # out-of-range brick and LOD are reported per request, the rest is served
    tc = srv.submit(np.array([1, n_bricks + 5, 2], np.uint32), np.array([0, 0, 9], np.uint8))
    rc, res = srv.poll(tc, timeout_us=10_000_000)
    assert rc == csgv.CSGV_OK
    assert [r.status for r in res] == [0, csgv.CSGV_ERR_RANGE, csgv.CSGV_ERR_RANGE]
    check_results(srv, v, [1], [0], res[:1])
    srv.release(tc)
    srv.close()
