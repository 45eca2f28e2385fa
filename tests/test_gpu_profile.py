"""The library's kernel timing (csgv_profile_*): events around each launch on the launching stream, a reserved
event pool, and read-and-clear semantics."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_profile_counts_each_launch_and_clears():
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((64, 64, 96), 40, seed=81, warp_amp=2, bg_permille=200)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    v = csgv.csgv_encode_bricks(d, 32, csgv.csgv_build_freq_table(d, 32, 1))
    n = v.info().n_bricks
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    lods = torch.zeros(n, dtype=torch.uint8, device="cuda")
    offs = torch.arange(n, dtype=torch.int64, device="cuda") * 32 ** 3
    out = torch.empty(n * 32 ** 3, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    csgv.profile_read()  # whatever an earlier test left
    csgv.profile_reserve(64)
    csgv.profile_enable(True)
    for _ in range(3):
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, st)
    csgv.profile_enable(False)
    csgv.csgv_decode_bricks(v, ids, lods, out, offs, st)  # not recorded
    prof = csgv.profile_read()
    assert set(prof) == {"rans_records", "rebuild"}, prof
    for name, (ms, launches) in prof.items():
        assert launches == 3 and 0.0 < ms < 1e3, (name, ms, launches)
    assert csgv.profile_read() == {}
    assert bool((st == 0).all())
    got = out.view(2, 2, 3, 32, 32, 32).permute(0, 3, 1, 4, 2, 5).reshape(64, 64, 96).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, vol)
    v.close()
