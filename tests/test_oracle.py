"""Pins of the CPU oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: expected values are the
hand-derived golden bricks (tests/golden), brute force on tiny bricks,
closed forms and invariants stated in the paper (Sec. 3.1-3.4), and
information-theoretic bounds on the rANS stage.
"""
import glob
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from tests import bruteforce as BF

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.txt")))


# ---------------------------------------------------------------- pyramid (Sec. 3.1)

def test_pyramid_node_count_closed_form():
    # sum_{l=0..N} (b/2^l)^3 = (8^(N+1) - 1) / 7; extra memory 14.3 % for b = 32 (Sec. 3.1, 3.4: "about 14%")
    for N in range(1, 7):
        assert O.pyramid_nodes(N) == (8 ** (N + 1) - 1) // 7
    extra = (O.pyramid_nodes(5) - 32 ** 3) / 32 ** 3
    assert abs(extra - 4681 / 32768) < 1e-12 and 0.14 < extra < 0.145


def test_pyramid_tie_goes_to_first_occurrence():
    # children (Morton order) A B B A C C D D: every label twice -> the first one, A (Sec. 3.4)
    kids = [5, 6, 6, 5, 7, 7, 8, 8]
    brick = np.zeros((2, 2, 2), np.uint32)
    for c, v in enumerate(kids):
        brick[(c >> 2) & 1, (c >> 1) & 1, c & 1] = v
    (l0, c0), (l1, c1) = O.pyramid(brick)
    assert l1[0, 0, 0] == 5 and c1[0, 0, 0] == 0
    # B first: B A A B ... -> B
    kids = [6, 5, 5, 6, 7, 7, 8, 8]
    for c, v in enumerate(kids):
        brick[(c >> 2) & 1, (c >> 1) & 1, c & 1] = v
    assert O.pyramid(brick)[1][0][0, 0, 0] == 6
    # strict majority beats first occurrence: A B B B C C D D -> B
    kids = [5, 6, 6, 6, 7, 7, 8, 8]
    for c, v in enumerate(kids):
        brick[(c >> 2) & 1, (c >> 1) & 1, c & 1] = v
    assert O.pyramid(brick)[1][0][0, 0, 0] == 6


@pytest.mark.parametrize("b,seed", [(4, 0), (8, 1), (16, 2)])
def test_pyramid_matches_bruteforce(b, seed):
    rng = np.random.default_rng(seed)
    for trial in range(4):
        brick = BF.voronoi_brick(rng, b, n_sites=3 + trial * 4, n_labels=2 + trial * 3)
        labs, csts = BF.mode_pyramid(brick)
        got = O.pyramid(brick)
        for l in range(len(labs)):
            assert np.array_equal(got[l][0], labs[l].astype(np.uint32)), l
            if l >= 1:
                assert np.array_equal(got[l][1].astype(bool), csts[l]), l


# ---------------------------------------------------------------- golden bricks (Sec. 3.2, Alg. 2)

@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p) for p in GOLDEN])
def test_golden_encoding(path):
    brick, palette, interior, leaf = BF.read_golden(path)
    pal, ni, nl = O.encode_brick(brick)
    assert pal.tolist() == palette
    assert ni.tolist() == interior
    assert nl.tolist() == leaf
    N = brick.shape[0].bit_length() - 1
    out, rc = O.decode_brick(pal, ni, nl, N, 0)
    assert rc == 0 and np.array_equal(out, brick)


def test_golden_covers_every_operation():
    seen = set()
    for path in GOLDEN:
        _, _, interior, leaf = BF.read_golden(path)
        for s in (interior, leaf):
            i = 0
            while i < len(s):
                op = s[i] & 7
                seen.add(op)
                i += 2 if op == 5 else 1
    assert seen == set(range(7))


# ---------------------------------------------------------------- round trips (Alg. 1 inverts Alg. 2)

def _roundtrip_all_lods(brick):
    N = brick.shape[0].bit_length() - 1
    pal, ni, nl = O.encode_brick(brick)
    labs, _ = BF.mode_pyramid(brick)
    for t in range(N + 1):
        out, rc = O.decode_brick(pal, ni, nl, N, t)
        assert rc == 0, (t, rc)
        assert np.array_equal(out, labs[t].astype(np.uint32)), t
    return pal, ni, nl


@pytest.mark.parametrize("k", [2, 3, 4])
def test_exhaustive_2cubed(k):
    # every 2^3 brick over k labels (k^8 bricks): decode(t=0) == brick, decode(t=1) == mode root
    for combo in itertools.product(range(k), repeat=8):
        brick = np.array(combo, np.uint32).reshape(2, 2, 2) * 3 + 1
        pal, ni, nl = O.encode_brick(brick)
        out, rc = O.decode_brick(pal, ni, nl, 1, 0)
        assert rc == 0 and np.array_equal(out, brick), combo
        root, rc = O.decode_brick(pal, ni, nl, 1, 1)
        labs, _ = BF.mode_pyramid(brick)
        assert rc == 0 and root[0, 0, 0] == labs[1][0, 0, 0]
        assert len(ni) == 0
        assert (len(nl) == 0) == (len(set(combo)) == 1)


def test_exhaustive_4cubed_constant_octants():
    # 3^8 bricks whose 2^3 octants are constant: every L1 node is constant, so only root children are coded,
    # all with the stop bit (Sec. 3.2 stop bits)
    for combo in itertools.product(range(3), repeat=8):
        brick = np.zeros((4, 4, 4), np.uint32)
        for c, v in enumerate(combo):
            dx, dy, dz = BF.CHILD[c]
            brick[2 * dz:2 * dz + 2, 2 * dy:2 * dy + 2, 2 * dx:2 * dx + 2] = v + 10
        pal, ni, nl = _roundtrip_all_lods(brick)
        assert len(nl) == 0
        if len(set(combo)) > 1:
            ops, i = [], 0
            while i < len(ni):
                ops.append(int(ni[i]))
                i += 2 if ni[i] & 7 == 5 else 1
            assert len(ops) == 8 and all((x >> 3) == 1 for x in ops)


@pytest.mark.parametrize("b", [4, 8, 16])
def test_random_voronoi_bricks_roundtrip_and_first_applicable(b):
    rng = np.random.default_rng(100 + b)
    n = {4: 300, 8: 120, 16: 25}[b]
    for i in range(n):
        brick = BF.voronoi_brick(rng, b, n_sites=int(rng.integers(1, 3 * b)), n_labels=int(rng.integers(1, 20)))
        pal, ni, nl = _roundtrip_all_lods(brick)
        if i % 4 == 0:
            assert BF.check_first_applicable(brick, pal, ni, nl) == []


def test_noise_bricks_palette_duplicates_and_deltas():
    # i.i.d. labels: many P_a, back references with delta up to 15, palette duplicates (Sec. 3.2 discussion)
    rng = np.random.default_rng(7)
    saw_big_delta = saw_dup = False
    for k in (3, 6, 17, 40):
        for _ in range(6):
            brick = rng.integers(0, k, size=(8, 8, 8)).astype(np.uint32)
            pal, ni, nl = _roundtrip_all_lods(brick)
            assert BF.check_first_applicable(brick, pal, ni, nl) == []
            saw_dup |= len(pal) > len(set(pal.tolist()))
            for s in (ni, nl):
                for j in range(len(s) - 1):
                    if s[j] & 7 == 5 and s[j + 1] >= 10:
                        saw_big_delta = True
    assert saw_dup and saw_big_delta


def test_homogeneous_brick_is_single_palette_entry():
    # Sec. 5 (CR histogram): a brick of one label costs one palette entry and no ops
    for b in (2, 4, 8, 16, 32):
        brick = np.full((b, b, b), 0xDEADBEEF, np.uint32)
        pal, ni, nl = O.encode_brick(brick)
        assert pal.tolist() == [0xDEADBEEF] and len(ni) == 0 and len(nl) == 0
        N = b.bit_length() - 1
        for t in range(N + 1):
            out, rc = O.decode_brick(pal, ni, nl, N, t)
            assert rc == 0 and (out == 0xDEADBEEF).all() and out.shape[0] == b >> t


def test_stream_invariants_on_structured_volume():
    rng = np.random.default_rng(11)
    for _ in range(20):
        brick = BF.voronoi_brick(rng, 16, n_sites=20, n_labels=12)
        pal, ni, nl, ops = O.encode_brick(brick, with_counts=True)
        # leaf stop bits are always 0 (Sec. 3.3); op code 7 never occurs; every P_a adds one palette entry
        i = 0
        while i < len(nl):
            assert nl[i] >> 3 == 0 and nl[i] & 7 != 7
            i += 2 if nl[i] & 7 == 5 else 1
        i = 0
        while i < len(ni):
            assert ni[i] & 7 != 7
            i += 2 if ni[i] & 7 == 5 else 1
        assert ops[6] == len(pal) - 1
        assert int(ops.sum()) + int(ops[5]) == len(ni) + len(nl)


def test_decoder_rejects_corrupt_streams():
    brick, palette, interior, leaf = BF.read_golden(
        os.path.join(os.path.dirname(__file__), "golden", "b4_delta_after_op.txt"))
    pal, ni, nl = O.encode_brick(brick)
    # invalid op code 7
    bad = nl.copy(); bad[1] = 7
    assert O.decode_brick(pal, ni, bad, 2, 0)[1] == O.ORC_ERR_CORRUPT
    # stop bit on a leaf
    bad = nl.copy(); bad[0] |= 8
    assert O.decode_brick(pal, ni, bad, 2, 0)[1] == O.ORC_ERR_CORRUPT
    # truncated leaf stream
    assert O.decode_brick(pal, ni, nl[:-3], 2, 0)[1] == O.ORC_ERR_CORRUPT
    # trailing symbols
    assert O.decode_brick(pal, ni, np.concatenate([nl, [0]]).astype(np.uint8), 2, 0)[1] == O.ORC_ERR_CORRUPT
    # P_delta reaching before palette[0]
    bad = nl.copy(); bad[10] = 15
    assert O.decode_brick(pal, ni, bad, 2, 0)[1] == O.ORC_ERR_CORRUPT
    # P_a past the end of the palette
    assert O.decode_brick(pal[:1], ni, nl, 2, 0)[1] == O.ORC_ERR_CORRUPT
    # neighbour outside the brick: R_x at child 1 of the first L1 parent (x = 1 -> +x parent is inside),
    # so use R_y at child 0 of the root's children on a 2^3 brick instead
    p2, i2, l2 = O.encode_brick(np.arange(8, dtype=np.uint32).reshape(2, 2, 2))
    bad = l2.copy(); bad[1] = 2
    assert O.decode_brick(p2, i2, bad, 1, 0)[1] == O.ORC_ERR_CORRUPT


# ---------------------------------------------------------------- frequency tables (Sec. 3.3, R11)

def test_normalize_sums_and_floors():
    rng = np.random.default_rng(3)
    for _ in range(200):
        counts = rng.integers(0, 10 ** rng.integers(1, 9), size=16).astype(np.uint64)
        counts[rng.random(16) < 0.3] = 0
        f = O.normalize(counts)
        assert f.sum() == 4096 and (f >= 1).all()
        # order preserving: more occurrences never get a smaller frequency
        for a in range(16):
            for c in range(16):
                if counts[a] > counts[c]:
                    assert f[a] >= f[c]
    assert O.normalize(np.zeros(16, np.uint64)).tolist() == [256] * 16
    one = np.zeros(16, np.uint64); one[8] = 12345
    f = O.normalize(one)
    assert f[8] == 4096 - 15 and f.sum() == 4096


TABLES = os.path.join(os.path.dirname(__file__), "golden", "tables")


def _read_golden(path):
    out = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split(":", 1)
            out[k.strip()] = [int(x, 0) for x in v.split()]
    return out


@pytest.mark.parametrize("name", ["normalize_tie_at_minimum", "normalize_tied_maxima", "normalize_large_counts"])
def test_normalize_hand_derived(name):
    # R11, worked by hand in tests/golden/tables: which symbols take the leftover units, ties to the lower symbol
    g = _read_golden(os.path.join(TABLES, name + ".txt"))
    counts = np.array(g["counts"], np.uint64)
    assert int(counts.sum()) == g["total"][0]
    floors = [1 + (c * 4080) // g["total"][0] for c in g["counts"]]  # exact Python integers
    assert 4096 - sum(floors) == g["leftover"][0]
    assert O.normalize(counts).tolist() == g["freq"]


def test_normalize_is_exact_near_the_top_of_the_domain():
    # counts whose product with 4080 passes 2^64; expected values from the closed form with exact integers
    c = np.zeros(16, np.uint64)
    c[0], c[5], c[15] = 2 ** 63, 2 ** 62, 2 ** 62 - 1  # total 2^64 - 1
    total = 2 ** 63 + 2 ** 62 + 2 ** 62 - 1
    f = O.normalize(c)
    assert f.sum() == 4096
    assert f[0] >= 1 + (2 ** 63 * 4080) // total and f[5] >= 1 + (2 ** 62 * 4080) // total
    assert f[0] <= 2 + (2 ** 63 * 4080) // total and f[5] <= 2 + (2 ** 62 * 4080) // total
    assert all(f[s] == 1 for s in range(16) if s not in (0, 5, 15))


def test_prepass_counts_the_nibbles_of_bricks_whose_id_is_a_multiple_of_stride():
    # R12 ("every s-th brick", Sec. 3.4): the prepass histogram equals the sum of the per-brick nibble
    # histograms of exactly the bricks with id % stride == 0, counted here brick by brick
    vol = _small_volume(seed=7, shape=(40, 36, 50), n_sites=60)  # 7 x 5 x 5 bricks of 8^3, padded
    b, N = 8, 3
    n = 7 * 5 * 5
    per = []
    for bid in range(n):
        _, ni, nl = O.encode_brick(_brick_of(vol, b, bid))
        per.append((np.bincount(ni, minlength=16), np.bincount(nl, minlength=16)))
    for stride in (1, 3, 7, 512):
        ids = [i for i in range(n) if i % stride == 0]
        want_i = sum(per[i][0] for i in ids)
        want_l = sum(per[i][1] for i in ids)
        ci, cl = O.count_nibbles(vol, N, stride=stride, n_threads=3)
        assert ci.tolist() == want_i.tolist() and cl.tolist() == want_l.tolist(), stride
    # the histograms of neighbouring offsets differ on this volume, so an offset slip cannot pass
    other = sum(per[i][1] for i in range(n) if i % 3 == 1)
    assert other.tolist() != sum(per[i][1] for i in range(n) if i % 3 == 0).tolist()


# ---------------------------------------------------------------- rANS (Sec. 3.3, R9, R10)

def _rand_freq(rng):
    counts = (rng.pareto(1.2, size=16) * 100).astype(np.uint64)
    return O.normalize(counts)


def _stream(rng, n, p):
    """n nibbles drawn from p, read as a stream (a P_delta op, op bits 5, is followed by its delta nibble);
    a P_delta op drawn as the very last nibble would lack its delta, so it becomes a P_0 op."""
    sym = rng.choice(16, size=n, p=p).astype(np.uint8)
    i = 0
    while i < n:
        if (sym[i] & 7) == 5:
            if i + 1 == n:
                sym[i] ^= 1
            i += 2
        else:
            i += 1
    return sym


def _state_counts(sym, K):
    """symbols per state under R10: op j and the delta of a P_delta op j on state j mod K"""
    n_k, i, j = [0] * K, 0, 0
    while i < len(sym):
        pd = (sym[i] & 7) == 5
        n_k[j % K] += 2 if pd else 1
        i += 2 if pd else 1
        j += 1
    return n_k


def test_rans_roundtrip_random():
    rng = np.random.default_rng(5)
    for _ in range(150):
        f = _rand_freq(rng)
        n = int(rng.integers(1, 3000))
        p = f / f.sum()
        sym = _stream(rng, n, p)
        K = int(rng.integers(1, min(32, n) + 1))
        w = O.rans_encode(sym, K, f)
        dec, rc = O.rans_decode(w, n, K, f)
        assert rc == 0 and np.array_equal(dec, sym)
        m = int(rng.integers(0, n + 1))
        pre, rc = O.rans_decode(w, n, K, f, m=m)
        assert rc == 0 and np.array_equal(pre, sym[:m])


def test_rans_uniform_table_is_four_bits_per_symbol():
    # f_s = 256 for all s: every symbol costs exactly 4 bits, so each state emits one 16-bit word per 4 of its
    # symbols and ends with a 32-bit flush: 2K + sum_k floor(n_k / 4) words (closed form), n_k the symbols
    # of state k
    f = np.full(16, 256, np.uint32)
    rng = np.random.default_rng(9)
    for n in (1, 3, 4, 5, 17, 100, 1001):
        for K in (1, 2, 5, min(32, n)):
            if K > n:
                continue
            sym = _stream(rng, n, np.full(16, 1 / 16))
            w = O.rans_encode(sym, K, f)
            n_k = _state_counts(sym, K)
            assert len(w) == 2 * K + sum(x // 4 for x in n_k), (n, K)


def test_rans_code_length_against_entropy():
    # static-table code length >= n * H(empirical) (Gibbs) and <= n * cross-entropy + flush/rounding slack
    rng = np.random.default_rng(13)
    for _ in range(30):
        f = _rand_freq(rng)
        n = int(rng.integers(2000, 20000))
        sym = _stream(rng, n, f / f.sum())
        K = int(rng.integers(1, 33))
        w = O.rans_encode(sym, K, f)
        bits = 16 * (len(w) - 2 * K)  # renormalisation words only
        cnt = np.bincount(sym, minlength=16)
        p = cnt[cnt > 0] / n
        H = -(p * np.log2(p)).sum()
        q = f / 4096.0
        CE = -(cnt * np.log2(q)).sum()
        assert bits + 32 * K >= n * H * (1 - 1e-3)
        assert bits <= CE + 0.005 * n + 48 * K


@pytest.mark.parametrize("name", ["rans_uniform_k2", "rans_uniform_k2_delta_last", "rans_uniform_k2_delta_word"])
def test_rans_hand_derived_stream(name):
    # R9/R10 worked by hand (tests/golden/tables/): op j on state j mod K, a delta on its op's state, per
    # step the ops then the deltas, final states low half first and state 0 first, renormalisation words in
    # coding order; the second file ends on a step whose one op is a P_delta, the third places a delta's
    # renormalisation word after that of the other state's op of its step
    g = _read_golden(os.path.join(TABLES, name + ".txt"))
    sym = np.array(g["symbols"], np.uint8)
    f = np.array(g["freq"], np.uint32)
    w = O.rans_encode(sym, g["K"][0], f)
    assert w.tolist() == g["words"]
    dec, rc = O.rans_decode(np.array(g["words"], np.uint16), len(sym), g["K"][0], f)
    assert rc == 0 and dec.tolist() == g["symbols"]


def test_rans_detects_wrong_final_state():
    rng = np.random.default_rng(17)
    f = _rand_freq(rng)
    sym = _stream(rng, 500, f / f.sum())
    w = O.rans_encode(sym, 4, f)
    bad = w.copy(); bad[0] ^= 0x10  # perturb a final state
    dec, rc = O.rans_decode(bad, 500, 4, f)
    assert rc == O.ORC_ERR_CORRUPT or not np.array_equal(dec, sym)
    dec, rc = O.rans_decode(np.concatenate([w, [1]]).astype(np.uint16), 500, 4, f)
    assert rc == O.ORC_ERR_CORRUPT  # unused trailing word


def test_lane_rule():
    assert O.lanes(0, 32, 256) == 0
    assert O.lanes(1, 32, 256) == 1
    assert O.lanes(511, 32, 256) == 1
    assert O.lanes(512, 32, 256) == 2
    assert O.lanes(10 ** 6, 32, 256) == 32
    assert O.lanes(10 ** 6, 1, 256) == 1


# ---------------------------------------------------------------- volume level (Sec. 3.1, 3.4)

def _small_volume(seed=1, shape=(40, 36, 50), n_sites=30):
    rng = np.random.default_rng(seed)
    Z, Y, X = shape
    sites = rng.integers(0, [X, Y, Z], size=(n_sites, 3))
    labels = rng.integers(1, 2 ** 32 - 1, size=n_sites, dtype=np.uint64).astype(np.uint32)
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    d = np.full(shape, np.iinfo(np.int64).max)
    vol = np.zeros(shape, np.uint32)
    for s in range(n_sites):
        ds = (x - sites[s, 0]) ** 2 + (y - sites[s, 1]) ** 2 + (z - sites[s, 2]) ** 2
        m = ds < d
        d[m] = ds[m]
        vol[m] = labels[s]
    return vol


def _brick_of(vol, b, bid):
    Z, Y, X = vol.shape
    nbx, nby = -(-X // b), -(-Y // b)
    bx, by, bz = bid % nbx, (bid // nbx) % nby, bid // (nbx * nby)
    zz = np.minimum(np.arange(bz * b, bz * b + b), Z - 1)
    yy = np.minimum(np.arange(by * b, by * b + b), Y - 1)
    xx = np.minimum(np.arange(bx * b, bx * b + b), X - 1)
    return vol[np.ix_(zz, yy, xx)]


@pytest.mark.parametrize("N", [2, 3, 4])
def test_volume_roundtrip_with_padding(N):
    vol = _small_volume()  # dims not multiples of b: clamp-to-edge padding (reading R8)
    b = 1 << N
    V = O.encode_volume(vol, N, stride=3, K_max=8, S_min=16)
    assert V.freq[:16].sum() == 4096 and V.freq[16:].sum() == 4096
    n = V.n_bricks
    ids = np.arange(n, dtype=np.uint32)
    for t in range(N + 1):
        out, off, st = O.decode_bricks(V, ids, np.full(n, t, np.uint8))
        assert (st == 0).all()
        B = b >> t
        for bid in range(0, n, max(1, n // 25)):
            got = out[int(off[bid]):int(off[bid]) + B ** 3].reshape(B, B, B)
            want = BF.mode_pyramid(_brick_of(vol, b, bid))[0][t].astype(np.uint32)
            assert np.array_equal(got, want), (bid, t)


def test_volume_mixed_requests_and_duplicates():
    vol = _small_volume(seed=2, shape=(32, 32, 32), n_sites=40)
    V = O.encode_volume(vol, 3, stride=1, K_max=32, S_min=32)
    rng = np.random.default_rng(4)
    ids = rng.integers(0, V.n_bricks, size=200).astype(np.uint32)
    lods = rng.integers(0, 4, size=200).astype(np.uint8)
    out, off, st = O.decode_bricks(V, ids, lods)
    assert (st == 0).all()
    for r in range(200):
        B = 8 >> int(lods[r])
        got = out[int(off[r]):int(off[r]) + B ** 3].reshape(B, B, B)
        want = BF.mode_pyramid(_brick_of(vol, 8, int(ids[r])))[0][int(lods[r])].astype(np.uint32)
        assert np.array_equal(got, want)
    # out-of-range brick id is reported per request
    _, _, st = O.decode_bricks(V, np.array([V.n_bricks], np.uint32), np.zeros(1, np.uint8))
    assert st[0] == O.ORC_ERR_ARG


def test_subsampled_prepass_barely_changes_cr():
    # Sec. 5: the compression ratio hardly changes with the prepass sampling stride
    import synth
    vol = synth.voronoi((128, 128, 128), 400, seed=21, warp_amp=4, bg_permille=300)
    full = O.encode_volume(vol, 4, stride=1)
    sub = O.encode_volume(vol, 4, stride=64)
    a, c = full.compressed_bytes(), sub.compressed_bytes()
    assert abs(a - c) / a < 0.01
    assert a <= c * 1.0005  # tables from all bricks fit the data at least as well


def test_decoded_bytes_are_multiples_of_lod_size():
    assert [(32 >> t) ** 3 for t in range(6)] == [32768, 4096, 512, 64, 8, 1]
    assert sum(8 ** k for k in range(6)) == O.pyramid_nodes(5)
    assert math.isclose(sum((32 >> t) ** 3 for t in range(6)) / 6, 6241.5)


def test_stream_edits_keep_the_grammar_and_the_oracle_total():
    """The stream editor of the GPU edit tests (tests/stream_mutants.py): parsing and flattening a real stream
    is the identity, and on its edits the oracle's decoder always returns labels from the palette or a corrupt
    status, never anything else (the edits reach both outcomes)."""
    import synth
    from tests import stream_mutants as SM
    base = synth.voronoi((16, 16, 16), 12, seed=11)
    pal, ni, nl = O.encode_brick(base)
    assert np.array_equal(SM.flatten(SM.parse(ni)), ni) and np.array_equal(SM.flatten(SM.parse(nl)), nl)
    seen = set()
    for e_i, e_l in SM.mutants(np.random.default_rng(5), ni, nl, 60):
        for t in range(5):
            lab, rc = O.decode_brick(pal, e_i, e_l, 4, t)
            assert rc in (O.ORC_OK, O.ORC_ERR_CORRUPT)
            if rc == O.ORC_OK:
                assert np.isin(lab, pal).all()
            seen.add(rc)
    assert seen == {O.ORC_OK, O.ORC_ERR_CORRUPT}
