"""The Worley-cell volume of the serving workload (2048 x 2048 x 1024 at full size).

The serving benchmark makes its 16 GB volume on the device (synth/gen_gpu.cu); the oracle's inputs come
from the host generator (synth/gen.c).  The two must make the same labels, and a Worley volume must
round-trip through the CUDA encoder and decoder exactly as through the oracle: byte-identical streams,
every LOD equal to the oracle's decode and LOD 0 equal to the volume (integer data, tolerance zero).
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

SHAPE = (96, 128, 144)  # z, y, x: 128 and 144 are not multiples of the 24-voxel cell, 144 not of 32


def test_worley_device_generator_equals_host_generator():
    host = synth.worley(SHAPE, 24, seed=4)
    dev = synth.worley_device(SHAPE, 24, seed=4)
    assert np.array_equal(dev.cpu().numpy().view(np.uint32), host)
    # a second seed and cell size, and an odd shape
    host = synth.worley((33, 70, 47), 11, seed=9)
    dev = synth.worley_device((33, 70, 47), 11, seed=9)
    assert np.array_equal(dev.cpu().numpy().view(np.uint32), host)


@pytest.mark.parametrize("b,stride", [(32, 7), (16, 1)])
def test_worley_roundtrip_against_oracle(b, stride):
    import torch
    import paper_2308_16619_b300 as csgv
    N = b.bit_length() - 1
    vol = synth.worley(SHAPE, 24, seed=4)
    d = synth.worley_device(SHAPE, 24, seed=4)
    V = O.encode_volume(vol, N, stride=stride)
    gv, t = csgv.csgv_encode_bricks_sampled(d, b, stride)
    e = gv.export()
    assert list(t.freq) == V.freq.tolist()
    for k in ("pal_off", "int_off", "leaf_off", "pal", "int_words", "leaf_words", "n_int_sym", "n_leaf_sym"):
        assert np.array_equal(e[k], getattr(V, k)), k
    n = V.n_bricks
    ids_h = np.arange(n, dtype=np.uint32)
    for lod in range(N + 1):
        lods_h = np.full(n, lod, np.uint8)
        offs_h, total = csgv.request_layout(b, lods_h)
        out = torch.full((total,), -1, dtype=torch.int32, device="cuda")
        st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        csgv.csgv_decode_bricks(gv, torch.from_numpy(ids_h.view(np.int32)).cuda(), torch.from_numpy(lods_h).cuda(),
                                out, torch.from_numpy(offs_h).cuda(), st)
        torch.cuda.synchronize()
        assert bool((st == 0).all())
        want, _, wst = O.decode_bricks(V, ids_h, lods_h)
        assert (wst == 0).all()
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want[:total]), lod
        if lod == 0:
            # reassemble the padded brick grid and compare with the volume itself
            Z, Y, X = SHAPE
            gx, gy, gz = -(-X // b), -(-Y // b), -(-Z // b)
            full = got.reshape(gz, gy, gx, b, b, b).transpose(0, 3, 1, 4, 2, 5).reshape(gz * b, gy * b, gx * b)
            assert np.array_equal(full[:Z, :Y, :X], vol)
    gv.close()
