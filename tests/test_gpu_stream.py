"""Streaming encoder (bricks fed in batches from a generator, the raw volume never whole) and the fiber
generator that feeds it: the device's bricks equal the host generator's volume, and the streamed volume is
byte-identical to the oracle's encode of that volume and to the one-call GPU encode."""
import numpy as np
import pytest

import oracle as O
import synth


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def assert_same_arrays(gpu, V):
    for k in ("freq", "pal_off", "int_off", "leaf_off", "pal", "int_words", "leaf_words", "n_int_sym", "n_leaf_sym"):
        assert np.array_equal(gpu[k], getattr(V, k)), k

pytestmark = pytest.mark.gpu

SHAPE = (64, 96, 128)  # z, y, x
CELL, TUBES, SEED = 32, 6, 9


def _bricks_of(vol, b):
    Z, Y, X = vol.shape
    return vol.reshape(Z // b, b, Y // b, b, X // b, b).transpose(0, 2, 4, 1, 3, 5).reshape(-1, b, b, b)


@pytest.fixture(scope="module")
def fiber_vol():
    return synth.fibers(SHAPE, CELL, TUBES, SEED)


@pytest.mark.parametrize("b", [32, 16])
def test_device_fiber_bricks_equal_host_volume(fiber_vol, b):
    import torch
    Z, Y, X = SHAPE
    n = (X // b) * (Y // b) * (Z // b)
    dev = synth.fiber_bricks_device((X, Y, Z), b, CELL, TUBES, SEED, first=0, m=n)
    got = dev.view(n, b, b, b).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, _bricks_of(fiber_vol, b))
    ids = torch.tensor([n - 1, 3, 0, 7], dtype=torch.int64, device="cuda")
    some = synth.fiber_bricks_device((X, Y, Z), b, CELL, TUBES, SEED, ids=ids).view(4, b, b, b).cpu().numpy()
    assert np.array_equal(some.view(np.uint32), _bricks_of(fiber_vol, b)[[n - 1, 3, 0, 7]])


@pytest.mark.parametrize("b,stride,batches", [(32, 2, (1, 2, 3)), (16, 5, (7, 1, 16, 24))])
def test_stream_encoder_equals_oracle_and_one_call(fiber_vol, b, stride, batches):
    import torch
    import paper_2308_16619_b300 as csgv
    Z, Y, X = SHAPE
    N = b.bit_length() - 1
    n = (X // b) * (Y // b) * (Z // b)
    # prepass over the sampled bricks only (ids multiple of stride), made on the device
    ids = torch.arange(0, n, stride, dtype=torch.int64, device="cuda")
    counts = csgv.csgv_count_bricks(synth.fiber_bricks_device((X, Y, Z), b, CELL, TUBES, SEED, ids=ids), b)
    table = csgv.csgv_freq_table_from_counts(counts)
    V = O.encode_volume(fiber_vol, N, stride=stride)
    assert np.array_equal(table.freq_array(), V.freq)
    enc = csgv.StreamEncoder((X, Y, Z), b, table)
    first, k = 0, 0
    while first < n:
        m = min(batches[k % len(batches)], n - first)
        enc.add(synth.fiber_bricks_device((X, Y, Z), b, CELL, TUBES, SEED, first=first, m=m), first)
        first += m
        k += 1
    v = enc.finish()
    torch.cuda.synchronize()
    assert_same_arrays(v.export(), V)
    one = csgv.csgv_encode_bricks(to_dev(fiber_vol), b, table)
    e1, e2 = one.export(), v.export()
    for key in e1:
        assert np.array_equal(e1[key], e2[key]), key
    # and it decodes to the volume
    ids32 = torch.arange(n, dtype=torch.int32, device="cuda")
    lods = torch.zeros(n, dtype=torch.uint8, device="cuda")
    offs = torch.arange(n, dtype=torch.int64, device="cuda") * b ** 3
    out = torch.empty(n * b ** 3, dtype=torch.int32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(v, ids32, lods, out, offs, status)
    assert bool((status == 0).all())
    assert np.array_equal(out.view(n, b, b, b).cpu().numpy().view(np.uint32), _bricks_of(fiber_vol, b))


def test_stream_encoder_rejects_out_of_order_and_unfinished():
    import paper_2308_16619_b300 as csgv
    b = 16
    table = csgv.csgv_freq_table_from_counts(np.arange(1, 33, dtype=np.uint64))
    enc = csgv.StreamEncoder((32, 32, 16), b, table)
    bricks = synth.fiber_bricks_device((32, 32, 16), b, 16, 2, 1, first=0, m=4)
    with pytest.raises(csgv.CsgvError):
        enc.add(bricks[: 2 * b ** 3], 1)  # expected brick 0 first
    enc.add(bricks[: 2 * b ** 3], 0)
    with pytest.raises(csgv.CsgvError):
        enc.finish()  # 2 of 4 bricks
    enc.add(bricks[2 * b ** 3:], 2)
    v = enc.finish()
    assert v.info().n_bricks == 4
