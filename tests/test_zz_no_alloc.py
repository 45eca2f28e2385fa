"""The allocation-free encoder entry point (csgv_encode_bricks_noalloc).

Some callers cannot allocate device memory: their GPU memory is owned by their
own pool allocator, or cudaFree's device-wide synchronisation would stall
their other work.  csgv_encode_bricks_noalloc encodes into output arrays the
caller provides, using a fixed scratch array inside the library.  These tests
call it through the C ABI and check that it produces exactly what the regular
csgv_encode_bricks produces (integer data: the tolerance is zero), on two
calls in a row (the shared scratch keeps the previous call's contents), and
that a volume too large for its scratch is refused with a clear message.

Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("b", [32, 64, 16, 8])
def test_noalloc_encoder_matches_allocating_encoder_on_two_calls(b):
    # 128^3: 64 bricks of 32^3, 8 of 64^3 (the level arrays carved from the scratch too), 512 of 16^3 and
    # 4096 of 8^3, each within the scratch's limit for its brick size
    import torch
    import synth
    import paper_2308_16619_b300 as csgv

    vol = synth.make("voronoi128")
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    table = csgv.csgv_build_freq_table(d, b, 1)
    ref_vol = csgv.csgv_encode_bricks(d, b, table)
    ref = ref_vol.export()
    n = len(ref["n_int_sym"])

    dev = dict(pal_off=torch.empty(n + 1, dtype=torch.int64, device="cuda"),
               pal=torch.empty(len(ref["pal"]) + 100, dtype=torch.int32, device="cuda"),
               int_off=torch.empty(n + 1, dtype=torch.int64, device="cuda"),
               int_words=torch.empty(len(ref["int_words"]) + 100, dtype=torch.int16, device="cuda"),
               leaf_off=torch.empty(n + 1, dtype=torch.int64, device="cuda"),
               leaf_words=torch.empty(len(ref["leaf_words"]) + 100, dtype=torch.int16, device="cuda"),
               n_int_sym=torch.empty(n, dtype=torch.int32, device="cuda"),
               n_leaf_sym=torch.empty(n, dtype=torch.int32, device="cuda"))
    for call in range(2):
        for t in dev.values():
            t.fill_(-1)  # stale contents must not leak into the result
        torch.cuda.synchronize()
        rc, totals = csgv.csgv_encode_bricks_noalloc(d, b, table, dev["pal_off"], dev["pal"], dev["int_off"],
                                                     dev["int_words"], dev["leaf_off"], dev["leaf_words"],
                                                     dev["n_int_sym"], dev["n_leaf_sym"])
        torch.cuda.synchronize()
        assert rc == csgv.CSGV_OK, csgv.lib().csgv_last_error()
        assert totals == [len(ref["pal"]), len(ref["int_words"]), len(ref["leaf_words"])]
        got = {k: v.cpu().numpy() for k, v in dev.items()}
        assert np.array_equal(got["pal_off"].view(np.uint64), ref["pal_off"])
        assert np.array_equal(got["int_off"].view(np.uint64), ref["int_off"])
        assert np.array_equal(got["leaf_off"].view(np.uint64), ref["leaf_off"])
        assert np.array_equal(got["pal"][:totals[0]].view(np.uint32), ref["pal"])
        assert np.array_equal(got["int_words"][:totals[1]].view(np.uint16), ref["int_words"])
        assert np.array_equal(got["leaf_words"][:totals[2]].view(np.uint16), ref["leaf_words"])
        assert np.array_equal(got["n_int_sym"].view(np.uint32), ref["n_int_sym"])
        assert np.array_equal(got["n_leaf_sym"].view(np.uint32), ref["n_leaf_sym"])
    ref_vol.close()


def test_noalloc_encoder_rejects_volumes_beyond_its_scratch():
    import torch
    import paper_2308_16619_b300 as csgv

    big = torch.zeros((224, 128, 128), dtype=torch.int32, device="cuda")  # 112 bricks of 32^3 > 99
    table = csgv.FreqTable()
    for i in range(32):
        table.freq[i] = 256
    off = torch.empty(113, dtype=torch.int64, device="cuda")
    small = torch.empty(112, dtype=torch.int32, device="cuda")
    rc, _ = csgv.csgv_encode_bricks_noalloc(big, 32, table, off, small, off.clone(), small.view(torch.int16),
                                            off.clone(), small.view(torch.int16), small.clone(), small.clone())
    assert rc == csgv.CSGV_ERR_INVALID_ARG
    msg = csgv.lib().csgv_last_error().decode()
    assert "112 bricks" in msg and "at most 99" in msg
    # output arrays that are too small are refused once the sizes are known, with the sizes reported
    vol = torch.zeros((64, 64, 64), dtype=torch.int32, device="cuda")
    vol[:, :, 17:] = 5
    t2 = csgv.csgv_build_freq_table(vol, 32, 1)
    off = torch.empty(9, dtype=torch.int64, device="cuda")
    tiny32 = torch.empty(1, dtype=torch.int32, device="cuda")
    tiny16 = torch.empty(1, dtype=torch.int16, device="cuda")
    cnt = torch.empty(8, dtype=torch.int32, device="cuda")
    rc, totals = csgv.csgv_encode_bricks_noalloc(vol, 32, t2, off, tiny32, off.clone(), tiny16, off.clone(), tiny16,
                                                 cnt, cnt.clone())
    torch.cuda.synchronize()
    assert rc == csgv.CSGV_ERR_INVALID_ARG and totals[0] > 1
    assert "too small" in csgv.lib().csgv_last_error().decode()
