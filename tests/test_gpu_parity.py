"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer codec, so the bar is bit-exact: decoded labels equal the oracle's
decode (and the original volume at LOD 0), GPU-encoded streams and tables are
byte-identical to the oracle's.
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _csgv():
    import paper_2308_16619_b300 as csgv
    return csgv


def to_dev(a):
    torch = _torch()
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    return torch.from_numpy(a).cuda()


def import_oracle_volume(V):
    csgv = _csgv()
    return csgv.csgv_volume_import(V.N, V.dims, V.K_max, V.S_min, V.freq, V.pal_off, V.pal, V.int_off, V.int_words,
                                   V.leaf_off, V.leaf_words, V.n_int_sym, V.n_leaf_sym)


def gpu_decode(volume, N, ids, lods, plain=False, offsets=None, total=None):
    torch = _torch()
    csgv = _csgv()
    ids = np.asarray(ids, np.uint32)
    lods = np.asarray(lods, np.uint8)
    if offsets is None:
        offsets, total = csgv.request_layout(1 << N, lods)
    out = torch.full((max(total, 1),), -1, dtype=torch.int32, device="cuda")
    status = torch.full((len(ids),), -99, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(volume, to_dev(ids), to_dev(lods), out, to_dev(np.asarray(offsets, np.int64)), status,
                            plain=plain)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32), np.asarray(offsets, np.int64), status.cpu().numpy()


def assert_same_arrays(gpu, V):
    assert np.array_equal(gpu["freq"], V.freq)
    for k in ("pal_off", "int_off", "leaf_off"):
        assert np.array_equal(gpu[k], getattr(V, k)), k
    for k in ("pal", "int_words", "leaf_words", "n_int_sym", "n_leaf_sym"):
        assert np.array_equal(gpu[k], getattr(V, k)), k


def structured_volume(seed, shape, n_sites, n_labels=None, warp=0, bg=0):
    if n_labels is None:
        return synth.voronoi(shape, n_sites, seed=seed, warp_amp=warp, bg_permille=bg)
    v = synth.voronoi(shape, n_sites, seed=seed, warp_amp=warp, bg_permille=bg)
    # fold labels into a small alphabet to force palette back references and duplicates
    u, inv = np.unique(v, return_inverse=True)
    return (inv.reshape(v.shape) % n_labels).astype(np.uint32) * 977 + 5


CASES = [
    # (name, shape zyx, b, sites, n_labels, K_max, S_min)
    ("b2", (6, 7, 9), 2, 12, 4, 32, 256),
    ("b4", (12, 16, 20), 4, 30, None, 4, 8),
    ("b8", (24, 40, 33), 8, 60, 9, 32, 16),
    ("b16", (48, 32, 64), 16, 80, None, 32, 64),
    ("b16_small_alphabet", (32, 48, 32), 16, 200, 5, 8, 32),
    ("b32", (64, 64, 96), 32, 120, None, 32, 256),
    ("b32_single_state", (64, 32, 64), 32, 200, 7, 1, 256),
    ("b32_many_states", (32, 64, 64), 32, 300, None, 32, 16),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_decode_oracle_streams_all_lods(case):
    name, shape, b, sites, nl, K_max, S_min = case
    N = b.bit_length() - 1
    vol = structured_volume(7, shape, sites, nl)
    V = O.encode_volume(vol, N, stride=1, K_max=K_max, S_min=S_min)
    gv = import_oracle_volume(V)
    n = V.n_bricks
    ids = np.repeat(np.arange(n, dtype=np.uint32), N + 1)
    lods = np.tile(np.arange(N + 1, dtype=np.uint8), n)
    out, off, st = gpu_decode(gv, N, ids, lods)
    ref, roff, rst = O.decode_bricks(V, ids, lods)
    assert (rst == 0).all()
    assert (st == 0).all(), np.unique(st, return_counts=True)
    assert np.array_equal(off, roff.astype(np.int64))
    assert np.array_equal(out[:len(ref)], ref)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gpu_encode_byte_identical(case):
    torch = _torch()
    csgv = _csgv()
    name, shape, b, sites, nl, K_max, S_min = case
    N = b.bit_length() - 1
    vol = structured_volume(11, shape, sites, nl)
    stride = 3
    V = O.encode_volume(vol, N, stride=stride, K_max=K_max, S_min=S_min)
    d = to_dev(vol)
    table = csgv.csgv_build_freq_table(d, b, stride)
    assert np.array_equal(table.freq_array(), V.freq)
    gv = csgv.csgv_encode_bricks(d, b, table, K_max=K_max, S_min=S_min)
    torch.cuda.synchronize()
    assert_same_arrays(gv.export(), V)


def test_prepass_counts_match_oracle():
    csgv = _csgv()
    vol = structured_volume(3, (64, 64, 64), 90)
    for N, stride in ((4, 1), (4, 5), (5, 2)):
        ci, cl = O.count_nibbles(vol, N, stride)
        t = csgv.csgv_build_freq_table(to_dev(vol), 1 << N, stride)
        assert np.array_equal(np.array(t.counts[:16], np.uint64), ci)
        assert np.array_equal(np.array(t.counts[16:], np.uint64), cl)


def test_voronoi128_roundtrip_and_streams():
    """128^3, 150 Voronoi cells, b = 32 (64 bricks), table from the whole volume."""
    torch = _torch()
    csgv = _csgv()
    vol = synth.make("voronoi128")
    V = O.encode_volume(vol, 5, stride=1)
    d = to_dev(vol)
    table = csgv.csgv_build_freq_table(d, 32, 1)
    gv = csgv.csgv_encode_bricks(d, 32, table)
    assert_same_arrays(gv.export(), V)
    n = V.n_bricks
    for t in range(6):
        ids = np.arange(n, dtype=np.uint32)
        out, off, st = gpu_decode(gv, 5, ids, np.full(n, t, np.uint8))
        ref, _, _ = O.decode_bricks(V, ids, np.full(n, t, np.uint8))
        assert (st == 0).all() and np.array_equal(out, ref), t
    # LOD 0 equals the original volume brick by brick
    out, off, st = gpu_decode(gv, 5, np.arange(n, dtype=np.uint32), np.zeros(n, np.uint8))
    bricks = out.reshape(4, 4, 4, 32, 32, 32)  # [bz, by, bx, z, y, x]
    rebuilt = bricks.transpose(0, 3, 1, 4, 2, 5).reshape(128, 128, 128)
    assert np.array_equal(rebuilt, vol)
    del torch


@pytest.mark.parametrize("b", [32, 16])
def test_voronoi512_full_roundtrip(b):
    """512^3 warped Voronoi, 30 % background: full GPU encode then decode, bit-exact against the volume;
    streams byte-identical to the oracle's on every brick."""
    torch = _torch()
    csgv = _csgv()
    N = b.bit_length() - 1
    vol = synth.make("voronoi512")
    d = to_dev(vol)
    table = csgv.csgv_build_freq_table(d, b, 512)
    gv = csgv.csgv_encode_bricks(d, b, table)
    V = O.encode_volume(vol, N, stride=512)
    assert_same_arrays(gv.export(), V)
    # the one-call encode the benchmark step runs (prepass counts from the encode's own nibbles of every
    # 512th brick): tables and streams byte-identical to the oracle's prepass-then-encode
    gs, ts = csgv.csgv_encode_bricks_sampled(d, b, 512)
    assert list(ts.freq) == V.freq.tolist()
    assert_same_arrays(gs.export(), V)
    gs.close()
    n = V.n_bricks
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    lods = torch.zeros(n, dtype=torch.uint8, device="cuda")
    offs = torch.arange(n, dtype=torch.int64, device="cuda") * b ** 3
    out = torch.empty(n * b ** 3, dtype=torch.int32, device="cuda")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    csgv.csgv_decode_bricks(gv, ids, lods, out, offs, status)
    g = 512 // b
    rebuilt = out.view(g, g, g, b, b, b).permute(0, 3, 1, 4, 2, 5).reshape(512, 512, 512)
    assert bool((status == 0).all())
    assert bool((rebuilt == d).all())


def test_plain_equals_batched_and_mixed_batch_equals_alone():
    vol = structured_volume(5, (64, 96, 64), 150, warp=0)
    V = O.encode_volume(vol, 5, stride=1)
    gv = import_oracle_volume(V)
    rng = np.random.default_rng(1)
    ids = rng.integers(0, V.n_bricks, size=300).astype(np.uint32)  # duplicates included
    lods = rng.integers(0, 6, size=300).astype(np.uint8)
    out, off, st = gpu_decode(gv, 5, ids, lods)
    outp, offp, stp = gpu_decode(gv, 5, ids, lods, plain=True)
    assert (st == 0).all() and (stp == 0).all()
    assert np.array_equal(out, outp)
    # each request decoded alone gives the same bytes as inside the mix; order does not matter
    perm = rng.permutation(300)
    outq, offq, stq = gpu_decode(gv, 5, ids[perm], lods[perm])
    for k, r in enumerate(perm[:60]):
        B3 = (32 >> int(lods[r])) ** 3
        alone, _, sa = gpu_decode(gv, 5, ids[r:r + 1], lods[r:r + 1])
        assert sa[0] == 0
        assert np.array_equal(alone[:B3], out[off[r]:off[r] + B3])
        assert np.array_equal(outq[offq[k]:offq[k] + B3], out[off[r]:off[r] + B3])


@pytest.mark.parametrize("b", [64, 32, 16])
def test_output_offsets_of_every_alignment(b):
    """Requests whose output starts 0, 4, 8 or 12 bytes past a 16-byte boundary (rows of four labels go out as
    one 16-byte, two 8-byte or four 4-byte stores; a constant brick's labels before the first and after the
    last 16-byte boundary one by one) decode to the oracle's labels at every LOD and leave the labels between
    requests untouched.  The volume has a homogeneous brick and a noise brick (many non-constant L1 nodes)."""
    N = b.bit_length() - 1
    vol = synth.voronoi((2 * b, 2 * b, 2 * b), 30, seed=71, warp_amp=2, bg_permille=300)
    vol[:b, :b, :b] = 17
    rng = np.random.default_rng(72)
    vol[b:, :b, :b] = rng.integers(0, 200, size=(b, b, b)).astype(np.uint32) + 3
    V = O.encode_volume(vol, N, stride=1)
    gv = import_oracle_volume(V)
    n = V.n_bricks
    ids = np.repeat(np.arange(n, dtype=np.uint32), N + 1)
    lods = np.tile(np.arange(N + 1, dtype=np.uint8), n)
    sizes = (b >> lods.astype(np.int64)) ** 3
    shift = (ids.astype(np.int64) + lods) % 4  # labels past the boundary: every residue at every LOD
    offsets = np.empty(len(ids), np.int64)
    end = 0
    for i in range(len(ids)):
        offsets[i] = -(-(end + 1) // 4) * 4 + shift[i]  # at least one untouched label before each request
        end = offsets[i] + sizes[i]
    total = int(end) + 1
    out, _, st = gpu_decode(gv, N, ids, lods, offsets=offsets, total=total)
    ref, roff, rst = O.decode_bricks(V, ids, lods)
    assert (st == 0).all() and (rst == 0).all()
    written = np.zeros(total, bool)
    for i in range(len(ids)):
        o, m, r = int(offsets[i]), int(sizes[i]), int(roff[i])
        assert np.array_equal(out[o:o + m], ref[r:r + m]), (i, int(ids[i]), int(lods[i]), int(shift[i]))
        written[o:o + m] = True
    assert (out[~written] == 0xFFFFFFFF).all()


def test_b32_bricks_with_many_non_constant_l1_nodes_take_the_full_layout():
    """32^3 bricks with uint8 palette indices decode in a compact leaf layout that holds at most 1280
    non-constant L1 nodes; bricks with more go to the full-layout kernel in the same decode call.  Here half
    the bricks are 8-label noise (every L1 node non-constant, small palettes), half are Voronoi cells, and
    some are mixed; every LOD of every brick, requests in shuffled order, against the oracle."""
    rng = np.random.default_rng(31)
    shape = (64, 64, 128)  # 2 x 2 x 4 bricks
    vol = structured_volume(3, shape, 40)
    noise = rng.integers(1, 9, size=shape).astype(np.uint32)
    vol[:, :, 64:] = noise[:, :, 64:]  # two brick columns of noise
    vol[:32, :32, 40:56] = noise[:32, :32, 40:56]  # part of one Voronoi brick
    V = O.encode_volume(vol, 5, stride=1)
    gv = import_oracle_volume(V)
    assert gv.info().max_palette <= 253
    # non-constant L1 nodes per brick, from the volume: some bricks above the compact layout's 1280
    n_nc = []
    for bid in range(V.n_bricks):
        bx, by, bz = bid % 4, (bid // 4) % 2, bid // 8
        br = vol[bz * 32:bz * 32 + 32, by * 32:by * 32 + 32, bx * 32:bx * 32 + 32]
        blocks = br.reshape(16, 2, 16, 2, 16, 2).transpose(0, 2, 4, 1, 3, 5).reshape(4096, 8)
        n_nc.append(int((blocks != blocks[:, :1]).any(axis=1).sum()))
    assert max(n_nc) > 1280 and min(n_nc) <= 1280
    n = V.n_bricks
    ids = np.repeat(np.arange(n, dtype=np.uint32), 6)
    lods = np.tile(np.arange(6, dtype=np.uint8), n)
    perm = rng.permutation(len(ids))
    ids, lods = ids[perm], lods[perm]
    out, off, st = gpu_decode(gv, 5, ids, lods)
    ref, roff, rst = O.decode_bricks(V, ids, lods)
    assert (rst == 0).all() and (st == 0).all(), np.unique(st, return_counts=True)
    assert np.array_equal(out[:len(ref)], ref)


def test_b32_leaf_minus_list_and_its_fallback():
    """The compact leaf layout resolves the -axis children of the leaf level from a list kept in the unused
    part of its children area, which holds 4 (1280 - listed nodes) entries; a brick with more -axis children
    resolves them per listed node instead.  Two 32^3 bricks of x-stripes (every L1 node of the striped part
    is non-constant, with three -axis children: R_y / R_z toward the previous node) over a constant
    background: the first striped in 10 of its 32 z-layers (1280 listed nodes, more -axis children than the
    list holds), the second in 4 (512 listed nodes, the list).  Every LOD against the oracle."""
    shape = (32, 32, 64)
    vol = np.full(shape, 7, np.uint32)
    x = np.arange(64)
    stripes = (1 + (x & 1)).astype(np.uint32)[None, None, :]
    vol[:10, :, :32] = np.broadcast_to(stripes[:, :, :32], (10, 32, 32))
    vol[:4, :, 32:] = np.broadcast_to(stripes[:, :, 32:], (4, 32, 32))
    V = O.encode_volume(vol, 5, stride=1)
    fits = []
    for bid in range(2):
        br = np.ascontiguousarray(vol[:, :, 32 * bid:32 * bid + 32])
        blocks = br.reshape(16, 2, 16, 2, 16, 2).transpose(0, 2, 4, 1, 3, 5).reshape(4096, 8)
        n_act = int((blocks != blocks[:, :1]).any(axis=1).sum())
        nl = list(O.encode_brick(br)[2])
        ops, i = [], 0
        while i < len(nl):
            ops.append(nl[i])
            i += 2 if (nl[i] & 7) == 5 else 1
        op = np.array(ops).reshape(-1, 8) & 7
        c = np.arange(8)
        minus = int((((op == 1) & ((c & 1) == 0)) | ((op == 2) & ((c & 2) == 0)) | ((op == 3) & ((c & 4) == 0))).sum())
        assert n_act <= 1280 and len(op) == n_act
        fits.append(minus <= 4 * (1280 - n_act))
    assert fits == [False, True]
    gv = import_oracle_volume(V)
    ids = np.repeat(np.arange(2, dtype=np.uint32), 6)
    lods = np.tile(np.arange(6, dtype=np.uint8), 2)
    out, off, st = gpu_decode(gv, 5, ids, lods)
    ref, roff, rst = O.decode_bricks(V, ids, lods)
    assert (rst == 0).all() and (st == 0).all()
    assert np.array_equal(out[:len(ref)], ref)


def test_wide_palette_path():
    """Bricks with more than 253 palette entries use 16-bit indices in shared memory."""
    rng = np.random.default_rng(2)
    vol = rng.integers(0, 5000, size=(32, 32, 64)).astype(np.uint32)
    vol[:, :, 32:] = 17  # one noise brick, one homogeneous brick
    V = O.encode_volume(vol, 5, stride=1)
    assert int(np.diff(V.pal_off.astype(np.int64)).max()) > 253
    gv = import_oracle_volume(V)
    assert gv.info().max_palette > 253
    ids = np.array([0, 1, 0, 1, 0], np.uint32)
    lods = np.array([0, 0, 1, 3, 5], np.uint8)
    out, off, st = gpu_decode(gv, 5, ids, lods)
    ref, _, _ = O.decode_bricks(V, ids, lods)
    assert (st == 0).all() and np.array_equal(out, ref)
    csgv = _csgv()
    d = to_dev(vol)
    t = csgv.csgv_build_freq_table(d, 32, 1)
    g2 = csgv.csgv_encode_bricks(d, 32, t)
    assert_same_arrays(g2.export(), V)


@pytest.mark.parametrize("N", [5, 4, 3])
def test_range_and_corrupt_status(N):
    """Statuses for bad ids and LODs, truncated streams, a cut palette and random word flips, with the
    one-stream-per-warp rANS kernel (b = 32) and the packed one (b <= 16); the other bricks stay exact."""
    vol = structured_volume(4, (32, 32, 64), 50)
    V = O.encode_volume(vol, N, stride=1)
    gv = import_oracle_volume(V)
    nb = V.n_bricks
    # out-of-range brick id and LOD
    out, off, st = gpu_decode(gv, N, [0, nb, 1, 0, 1], [0, 0, 0, N + 1, N])
    assert st.tolist() == [0, 7, 0, 7, 0]
    csgv = _csgv()
    ids = np.array([0, 1], np.uint32)
    lods = np.zeros(2, np.uint8)
    # truncated leaf stream of brick 0: fewer words than its symbols need
    lo = V.leaf_off.copy()
    lw = np.delete(V.leaf_words, np.arange(int(lo[1]) - 5, int(lo[1])))
    lo[1:] -= 5
    bad = csgv.csgv_volume_import(N, V.dims, V.K_max, V.S_min, V.freq, V.pal_off, V.pal, V.int_off, V.int_words, lo,
                                  lw, V.n_int_sym, V.n_leaf_sym)
    out, off, st = gpu_decode(bad, N, ids, lods)
    ref, _, _ = O.decode_bricks(V, ids, lods)
    assert st[0] == 4 and st[1] == 0
    assert np.array_equal(out[off[1]:], ref[off[1]:])
    # palette of brick 0 cut to one entry: P_a runs past the palette
    po = V.pal_off.copy()
    cut = int(po[1]) - 1
    pal = np.delete(V.pal, np.arange(1, 1 + cut))
    po[1:] -= cut
    bad = csgv.csgv_volume_import(N, V.dims, V.K_max, V.S_min, V.freq, po, pal, V.int_off, V.int_words, V.leaf_off,
                                  V.leaf_words, V.n_int_sym, V.n_leaf_sym)
    out, off, st = gpu_decode(bad, N, ids, lods)
    assert st[0] == 4 and st[1] == 0
    # random word flips: never a fault; untouched bricks stay exact
    rng = np.random.default_rng(8)
    for trial in range(5):
        iw = V.int_words.copy()
        lw = V.leaf_words.copy()
        k = rng.integers(int(V.int_off[0]), int(V.int_off[1]), size=3)
        iw[k] ^= rng.integers(1, 65535, size=3).astype(np.uint16)
        k = rng.integers(int(V.leaf_off[0]), int(V.leaf_off[1]), size=3)
        lw[k] ^= rng.integers(1, 65535, size=3).astype(np.uint16)
        bad = csgv.csgv_volume_import(N, V.dims, V.K_max, V.S_min, V.freq, V.pal_off, V.pal, V.int_off, iw,
                                      V.leaf_off, lw, V.n_int_sym, V.n_leaf_sym)
        out, off, st = gpu_decode(bad, N, ids, lods)
        assert st[0] in (0, 4) and st[1] == 0
        assert np.array_equal(out[off[1]:], ref[off[1]:])


def test_one_table_and_single_state_variants_round_trip():
    """Coding variants (one table for both streams; K_max = 1, the paper's single rANS state) decode exactly."""
    import torch
    import paper_2308_16619_b300 as csgv
    vol = synth.voronoi((64, 96, 128), 120, seed=31, warp_amp=4, bg_permille=300)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    two = csgv.csgv_build_freq_table(d, 16, 1)
    c = np.array(two.counts[:], np.uint64)
    one = csgv.csgv_freq_table_from_counts(np.concatenate([c[:16] + c[16:], c[:16] + c[16:]]))
    assert one.freq[:16] == one.freq[16:]
    for table, km in ((one, 32), (two, 1)):
        v = csgv.csgv_encode_bricks(d, 16, table, K_max=km)
        n = v.info().n_bricks
        out = torch.empty(n * 16 ** 3, dtype=torch.int32, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        csgv.csgv_decode_bricks(v, torch.arange(n, dtype=torch.int32, device="cuda"),
                                torch.zeros(n, dtype=torch.uint8, device="cuda"), out,
                                torch.arange(n, dtype=torch.int64, device="cuda") * 16 ** 3, st)
        torch.cuda.synchronize()
        assert bool((st == 0).all())
        got = out.cpu().numpy().view(np.uint32).reshape(4, 6, 8, 16, 16, 16).transpose(0, 3, 1, 4, 2, 5)
        assert np.array_equal(got.reshape(vol.shape), vol)
        v.close()


@pytest.mark.parametrize("b,shape,stride", [(32, (128, 128, 128), 1), (32, (128, 128, 128), 5),
                                            (2, (64, 64, 128), 512)])
def test_sampled_encode_equals_prepass_then_encode(b, shape, stride):
    """csgv_encode_bricks_sampled (tables from the encode's own nibbles of every stride-th brick) gives the
    same tables and byte-identical streams as csgv_build_freq_table followed by csgv_encode_bricks; the
    2^3 case has more bricks than one encode batch and takes the two-call path inside."""
    import torch
    csgv = _csgv()
    vol = synth.voronoi(shape, 300, seed=37, warp_amp=4, bg_permille=300)
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    t1 = csgv.csgv_build_freq_table(d, b, stride)
    v1 = csgv.csgv_encode_bricks(d, b, t1)
    v2, t2 = csgv.csgv_encode_bricks_sampled(d, b, stride)
    assert list(t1.freq) == list(t2.freq) and list(t1.counts) == list(t2.counts)
    e1, e2 = v1.export(), v2.export()
    for k in e1:
        assert np.array_equal(e1[k], e2[k]), k
    v1.close()
    v2.close()


@pytest.mark.parametrize("kind", ["constant", "halves", "stripes"])
def test_sampled_tables_degenerate_counts(kind):
    """Tables normalised on the device from sampled counts equal the host normalisation when the counts
    are all zero (constant volume: uniform tables) or concentrated on one or two symbols (many zero-count
    ties, leftover units going to the largest counts)."""
    import torch
    csgv = _csgv()
    vol = np.full((64, 64, 64), 7, np.uint32)
    if kind == "halves":
        vol[:, :, 37:] = 9
    elif kind == "stripes":
        vol[:, :, ::2] = 3
    d = torch.from_numpy(vol.view(np.int32)).cuda()
    t1 = csgv.csgv_build_freq_table(d, 32, 1)
    v2, t2 = csgv.csgv_encode_bricks_sampled(d, 32, 1)
    hostt = csgv.csgv_freq_table_from_counts(list(t1.counts))
    assert list(t1.freq) == list(hostt.freq) == list(t2.freq)
    if kind == "constant":
        assert list(t2.freq) == [256] * 32
    v2.close()


def test_destroy_async_then_reuse_memory():
    """A volume freed in stream order right after its decode is queued decodes correctly, and a volume
    encoded next (reusing the freed pool memory) decodes correctly too."""
    import torch
    csgv = _csgv()
    outs = []
    for seed in (41, 42, 43):
        vol = synth.voronoi((64, 64, 96), 150, seed=seed, warp_amp=3, bg_permille=200)
        d = torch.from_numpy(vol.view(np.int32)).cuda()
        v, _ = csgv.csgv_encode_bricks_sampled(d, 16, 3)
        n = v.info().n_bricks
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        lods = torch.zeros(n, dtype=torch.uint8, device="cuda")
        offs = torch.arange(n, dtype=torch.int64, device="cuda") * 16 ** 3
        out = torch.empty(n * 16 ** 3, dtype=torch.int32, device="cuda")
        status = torch.empty(n, dtype=torch.int32, device="cuda")
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
        v.close_async()
        outs.append((vol, out, status))
    torch.cuda.synchronize()
    for vol, out, status in outs:
        assert bool((status == 0).all())
        got = out.view(-1, 16, 16, 16).cpu().numpy().view(np.uint32)
        bz, by, bx = (s // 16 for s in vol.shape)
        want = vol.reshape(bz, 16, by, 16, bx, 16).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 16, 16, 16)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("block,n_labels", [(8, 18), (8, 23), (8, 40), (4, 23), (2, 19)])
def test_palette_churn_byte_identical(block, n_labels):
    """Blocks of block^3 voxels with labels drawn from 18-40 values: many palette ops per brick, labels that
    leave the 17-entry window and come back, and P_delta at every depth; the encoder's streams are
    byte-identical to the oracle's (8^3 blocks: up to a few hundred palette children per brick, 4^3 and
    2^3: thousands)."""
    torch = _torch()
    csgv = _csgv()
    rng = np.random.default_rng(block * 100 + n_labels)
    shape = (32, 32, 64)
    g = rng.integers(0, n_labels, size=(shape[0] // block, shape[1] // block, shape[2] // block))
    vol = np.repeat(np.repeat(np.repeat(g, block, 0), block, 1), block, 2).astype(np.uint32) * 131 + 9
    V = O.encode_volume(vol, 5, stride=1)
    d = to_dev(vol)
    t = csgv.csgv_build_freq_table(d, 32, 1)
    assert np.array_equal(t.freq_array(), V.freq)
    gv = csgv.csgv_encode_bricks(d, 32, t)
    torch.cuda.synchronize()
    assert_same_arrays(gv.export(), V)


@pytest.mark.parametrize("kind", ["voronoi", "small_alphabet", "noise_and_constant", "thousand_labels"])
def test_b64_encode_byte_identical_and_decode_all_lods(kind):
    """b = 64 (the level arrays in global memory on both sides): GPU streams byte-identical to the oracle's,
    and every brick at every LOD 0..6 decodes to the oracle's labels.  The decoder keeps the levels as uint8,
    uint16 or uint32 palette indices by the largest palette: the noise brick's palette (about 200 000 labels)
    is past 2^16 entries, the thousand-label brick's past 253."""
    csgv = _csgv()
    if kind == "voronoi":
        vol = synth.voronoi((64, 128, 192), 90, seed=61, warp_amp=3, bg_permille=250)
    elif kind == "small_alphabet":
        vol = structured_volume(62, (128, 64, 64), 150, 6)
    elif kind == "noise_and_constant":
        rng = np.random.default_rng(63)
        vol = np.full((64, 64, 128), 41, np.uint32)
        vol[:, :, :64] = rng.integers(0, 1 << 30, size=(64, 64, 64)).astype(np.uint32)
    else:
        vol = synth.voronoi((64, 64, 128), 90, seed=66, warp_amp=2, bg_permille=100)
        rng = np.random.default_rng(67)
        vol[20:44, 20:44, 20:44] = rng.integers(0, 1000, size=(24, 24, 24)).astype(np.uint32) + 7
    V = O.encode_volume(vol, 6, stride=1)
    d = to_dev(vol)
    t = csgv.csgv_build_freq_table(d, 64, 1)
    assert np.array_equal(t.freq_array(), V.freq)
    gv = csgv.csgv_encode_bricks(d, 64, t)
    assert_same_arrays(gv.export(), V)
    if kind == "noise_and_constant":
        assert gv.info().max_palette > 65536
    if kind == "thousand_labels":
        assert 253 < gv.info().max_palette <= 65533
    n = V.n_bricks
    ids = np.repeat(np.arange(n, dtype=np.uint32), 7)
    lods = np.tile(np.arange(7, dtype=np.uint8), n)
    out, off, st = gpu_decode(gv, 6, ids, lods)
    ref, roff, rst = O.decode_bricks(V, ids, lods)
    assert (rst == 0).all() and (st == 0).all(), np.unique(st, return_counts=True)
    assert np.array_equal(out[:len(ref)], ref)


def test_b64_range_and_corrupt_status():
    """The b = 64 rebuild (levels in the workspace) reports the same statuses as the shared-memory kernel:
    range errors for a bad id or LOD, corrupt for a truncated stream or a cut palette, and random word
    flips never touch the other bricks of the batch."""
    csgv = _csgv()
    vol = synth.voronoi((64, 64, 128), 60, seed=64, warp_amp=2, bg_permille=200)
    V = O.encode_volume(vol, 6, stride=1)
    gv = import_oracle_volume(V)
    out, off, st = gpu_decode(gv, 6, [0, 2, 1, 0, 1], [0, 0, 0, 7, 6])
    assert st.tolist() == [0, 7, 0, 7, 0]
    ids = np.array([0, 1], np.uint32)
    lods = np.zeros(2, np.uint8)
    ref, _, _ = O.decode_bricks(V, ids, lods)
    lo = V.leaf_off.copy()
    lw = np.delete(V.leaf_words, np.arange(int(lo[1]) - 5, int(lo[1])))
    lo[1:] -= 5
    bad = csgv.csgv_volume_import(6, V.dims, V.K_max, V.S_min, V.freq, V.pal_off, V.pal, V.int_off, V.int_words, lo,
                                  lw, V.n_int_sym, V.n_leaf_sym)
    out, off, st = gpu_decode(bad, 6, ids, lods)
    assert st[0] == 4 and st[1] == 0
    assert np.array_equal(out[off[1]:], ref[off[1]:])
    po = V.pal_off.copy()
    cut = int(po[1]) - 1
    pal = np.delete(V.pal, np.arange(1, 1 + cut))
    po[1:] -= cut
    bad = csgv.csgv_volume_import(6, V.dims, V.K_max, V.S_min, V.freq, po, pal, V.int_off, V.int_words, V.leaf_off,
                                  V.leaf_words, V.n_int_sym, V.n_leaf_sym)
    out, off, st = gpu_decode(bad, 6, ids, lods)
    assert st[0] == 4 and st[1] == 0
    assert np.array_equal(out[off[1]:], ref[off[1]:])
    rng = np.random.default_rng(65)
    for trial in range(4):
        iw = V.int_words.copy()
        lw = V.leaf_words.copy()
        k = rng.integers(int(V.int_off[0]), int(V.int_off[1]), size=3)
        iw[k] ^= rng.integers(1, 65535, size=3).astype(np.uint16)
        k = rng.integers(int(V.leaf_off[0]), int(V.leaf_off[1]), size=3)
        lw[k] ^= rng.integers(1, 65535, size=3).astype(np.uint16)
        bad = csgv.csgv_volume_import(6, V.dims, V.K_max, V.S_min, V.freq, V.pal_off, V.pal, V.int_off, iw,
                                      V.leaf_off, lw, V.n_int_sym, V.n_leaf_sym)
        out, off, st = gpu_decode(bad, 6, ids, lods)
        assert st[0] in (0, 4) and st[1] == 0
        assert np.array_equal(out[off[1]:], ref[off[1]:])


@pytest.mark.parametrize("b", [32, 16, 8])
def test_edited_op_streams_decode_like_the_oracle(b):
    """Random edits of one brick's op streams (reuse ops exchanged, P_delta inserted, removed or given another
    delta, P_a added or dropped, op 7, stop bits set or flipped; tests/stream_mutants.py), each edited pair
    rANS-coded with the oracle's coder into a brick of its own: at every LOD the CUDA decoder either gives the
    labels the oracle decodes from the edited nibbles (Alg. 1) or, exactly when the oracle rejects them,
    status 4.  The edits reach op combinations the encoder never emits (R_a toward +axis next to P_delta, P_a
    runs, deltas past the palette), so this pins the byte-wise 8-children decode of the rebuild against the
    oracle's one child at a time."""
    from tests import stream_mutants as SM
    N = b.bit_length() - 1
    base = synth.voronoi((b, b, b), 40 if b == 32 else 12, seed=11)
    pal, ni, nl = O.encode_brick(base)
    V = O.encode_volume(base, N, stride=1)
    freq = np.asarray(V.freq, np.uint32)
    rng = np.random.default_rng(100 + b)
    edits = [(ni, nl)] + SM.mutants(rng, ni, nl, 63)
    M = len(edits)
    pal_off = np.arange(M + 1, dtype=np.uint64) * len(pal)
    int_w, leaf_w, int_off, leaf_off, nis, nls = [], [], [0], [0], [], []
    for e_i, e_l in edits:
        wi = O.rans_encode(e_i, O.lanes(len(e_i), 32, 256), freq[:16]) if len(e_i) else np.zeros(0, np.uint16)
        wl = O.rans_encode(e_l, O.lanes(len(e_l), 32, 256), freq[16:]) if len(e_l) else np.zeros(0, np.uint16)
        int_w.append(wi)
        leaf_w.append(wl)
        int_off.append(int_off[-1] + len(wi))
        leaf_off.append(leaf_off[-1] + len(wl))
        nis.append(len(e_i))
        nls.append(len(e_l))
    csgv = _csgv()
    gv = csgv.csgv_volume_import(N, (b * M, b, b), 32, 256, freq, pal_off, np.tile(pal, M),
                                 np.asarray(int_off, np.uint64), np.concatenate(int_w).astype(np.uint16),
                                 np.asarray(leaf_off, np.uint64), np.concatenate(leaf_w).astype(np.uint16),
                                 np.asarray(nis, np.uint32), np.asarray(nls, np.uint32))
    valid = 0
    for t in range(N + 1):
        out, off, st = gpu_decode(gv, N, np.arange(M, dtype=np.uint32), np.full(M, t, np.uint8))
        for m, (e_i, e_l) in enumerate(edits):
            ref, rc = O.decode_brick(pal, e_i, e_l, N, t)
            if rc == O.ORC_OK:
                valid += t == 0
                assert st[m] == 0, (t, m, st[m])
                assert np.array_equal(out[off[m]:off[m] + ref.size], ref.ravel()), (t, m)
            else:
                assert rc == O.ORC_ERR_CORRUPT and st[m] == 4, (t, m, rc, st[m])
    assert 10 <= valid < M  # both outcomes are exercised
