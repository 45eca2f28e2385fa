"""Plain CPU oracle of the compressed segmentation volume brick codec.

TEST INFRASTRUCTURE ONLY: imported by the tests, by __graft_entry__.smoke()
and by the CPU-baseline leg of bench.py.  The product path (the CUDA library
and its binding) never imports it, and it never imports the product path.

Thin ctypes wrapper over csgv_oracle.c; all arithmetic lives in the C file,
which follows the paper step by step (Sec. 3.1-3.4, Alg. 1 and Alg. 2).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

ORC_OK, ORC_ERR_ARG, ORC_ERR_CORRUPT, ORC_ERR_NOMEM = 0, 1, 2, 3
OPS = ("R_p", "R_x", "R_y", "R_z", "P_0", "P_delta", "P_a")

_lib = None


def lib():
    global _lib
    if _lib is None:
        # CSGV_ORACLE_LIB points the tests at another build of csgv_oracle.c (the planted-mistake
        # copies of tests/test_oracle_mutants.py); by default the library built from this directory
        _lib = C.CDLL(os.environ.get("CSGV_ORACLE_LIB") or _build.build())
        u64p = C.POINTER(C.c_uint64)
        _lib.csgvo_pyramid_nodes.restype = C.c_uint64
        _lib.csgvo_pyramid_nodes.argtypes = [C.c_int]
        _lib.csgvo_encode_volume.restype = C.c_void_p
        _lib.csgvo_encode_volume.argtypes = [C.c_void_p, u64p, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32,
                                             C.c_void_p, C.c_int, C.POINTER(C.c_int)]
        _lib.csgvo_volume_free.argtypes = [C.c_void_p]
        _lib.csgvo_volume_sizes.argtypes = [C.c_void_p, u64p]
        _lib.csgvo_volume_tables.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.csgvo_volume_export.argtypes = [C.c_void_p] + [C.c_void_p] * 8
        _lib.csgvo_lanes.restype = C.c_uint32
        _lib.csgvo_lanes.argtypes = [C.c_uint32] * 3
        _lib.csgvo_decode_bricks.argtypes = [C.c_int, C.c_uint32, C.c_uint32, C.c_void_p, C.c_uint64] + \
            [C.c_void_p] * 10 + [C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        _lib.csgvo_count_nibbles.argtypes = [C.c_void_p, u64p, C.c_int, C.c_uint64, C.c_int, C.c_void_p,
                                             C.c_void_p]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _u64x3(dims):
    return (C.c_uint64 * 3)(*[int(d) for d in dims])


def default_threads():
    return max(1, os.cpu_count() or 1)


def pyramid_nodes(N):
    return int(lib().csgvo_pyramid_nodes(N))


def level_offsets(N):
    """Offsets of levels 0..N (+ total) in the concatenated pyramid arrays."""
    offs, o = [], 0
    for l in range(N + 1):
        offs.append(o)
        o += (1 << (N - l)) ** 3
    offs.append(o)
    return offs


def pyramid(brick):
    """Sec. 3.1: list of (labels, const) per level l = 0..N, each shaped (B,B,B) indexed [z,y,x]."""
    brick = np.ascontiguousarray(brick, dtype=np.uint32)
    b = brick.shape[0]
    N = b.bit_length() - 1
    n = pyramid_nodes(N)
    lab = np.zeros(n, np.uint32)
    cst = np.zeros(n, np.uint8)
    rc = lib().csgvo_pyramid(_p(brick), N, _p(lab), _p(cst))
    assert rc == 0, rc
    offs = level_offsets(N)
    out = []
    for l in range(N + 1):
        B = b >> l
        out.append((lab[offs[l]:offs[l + 1]].reshape(B, B, B), cst[offs[l]:offs[l + 1]].reshape(B, B, B)))
    return out


def encode_brick(brick, with_counts=False):
    """Alg. 2 on one brick: (palette, interior nibbles, leaf nibbles[, op counts])."""
    brick = np.ascontiguousarray(brick, dtype=np.uint32)
    b = brick.shape[0]
    N = b.bit_length() - 1
    nodes = pyramid_nodes(N)
    pal = np.zeros(nodes, np.uint32)
    ni = np.zeros(2 * (nodes - b ** 3) + 1, np.uint8)
    nl = np.zeros(2 * b ** 3, np.uint8)
    npal, nint, nleaf = C.c_uint32(), C.c_uint32(), C.c_uint32()
    ops = np.zeros(7, np.uint64)
    rc = lib().csgvo_encode_brick(_p(brick), N, _p(pal), C.c_uint32(nodes), C.byref(npal), _p(ni),
                                  C.c_uint32(len(ni)), C.byref(nint), _p(nl), C.c_uint32(len(nl)),
                                  C.byref(nleaf), _p(ops))
    assert rc == 0, rc
    res = (pal[:npal.value].copy(), ni[:nint.value].copy(), nl[:nleaf.value].copy())
    return res + (ops,) if with_counts else res


def decode_brick(palette, int_nib, leaf_nib, N, t):
    """Alg. 1: returns ((b>>t)^3 labels shaped [z,y,x], rc)."""
    palette = np.ascontiguousarray(palette, np.uint32)
    int_nib = np.ascontiguousarray(int_nib, np.uint8)
    leaf_nib = np.ascontiguousarray(leaf_nib, np.uint8)
    B = (1 << N) >> t
    out = np.zeros(B ** 3, np.uint32)
    rc = lib().csgvo_decode_brick(_p(palette), C.c_uint32(len(palette)), _p(int_nib), C.c_uint32(len(int_nib)),
                                  _p(leaf_nib), C.c_uint32(len(leaf_nib)), N, t, _p(out))
    return out.reshape(B, B, B), rc


def normalize(counts):
    """Sec. 3.3 / reading R11: 16 counts -> 16 frequencies summing to 4096."""
    counts = np.ascontiguousarray(counts, np.uint64)
    freq = np.zeros(16, np.uint32)
    lib().csgvo_normalize(_p(counts), _p(freq))
    return freq


def lanes(n, K_max, S_min):
    return int(lib().csgvo_lanes(n, K_max, S_min))


def rans_encode(sym, K, freq):
    sym = np.ascontiguousarray(sym, np.uint8)
    freq = np.ascontiguousarray(freq, np.uint32)
    cap = 2 * K + len(sym) + 2
    words = np.zeros(cap, np.uint16)
    nw = C.c_uint32()
    rc = lib().csgvo_rans_encode(_p(sym), C.c_uint32(len(sym)), C.c_uint32(K), _p(freq), _p(words),
                                 C.c_uint32(cap), C.byref(nw))
    assert rc == 0, rc
    return words[:nw.value].copy()


def rans_decode(words, n, K, freq, m=None):
    words = np.ascontiguousarray(words, np.uint16)
    freq = np.ascontiguousarray(freq, np.uint32)
    m = n if m is None else m
    sym = np.zeros(max(m, 1), np.uint8)
    rc = lib().csgvo_rans_decode(_p(words), C.c_uint32(len(words)), C.c_uint32(n), C.c_uint32(m),
                                 C.c_uint32(K), _p(freq), _p(sym))
    return sym[:m], rc


def count_nibbles(vol, N, stride=1, n_threads=None):
    """Prepass (Sec. 3.4): nibble counts of interior and leaf streams over every stride-th brick."""
    vol = np.ascontiguousarray(vol, np.uint32)
    ci = np.zeros(16, np.uint64)
    cl = np.zeros(16, np.uint64)
    Z, Y, X = vol.shape
    rc = lib().csgvo_count_nibbles(_p(vol), _u64x3((X, Y, Z)), N, stride, n_threads or default_threads(),
                                   _p(ci), _p(cl))
    assert rc == 0, rc
    return ci, cl


class Volume:
    """Concatenated per-brick arrays of an encoded volume (host numpy arrays).

    Field layout (shared by construction with the CUDA library's export):
    pal_off/int_off/leaf_off are exclusive prefix sums with n_bricks+1
    entries; words are uint16; freq = interior table then leaf table.
    """

    def __init__(self, N, dims, K_max, S_min, freq, pal_off, pal, int_off, int_words, leaf_off, leaf_words,
                 n_int_sym, n_leaf_sym, op_counts=None):
        self.N, self.dims, self.K_max, self.S_min = N, tuple(int(d) for d in dims), K_max, S_min
        self.freq = np.ascontiguousarray(freq, np.uint32)
        self.pal_off, self.pal = pal_off, pal
        self.int_off, self.int_words = int_off, int_words
        self.leaf_off, self.leaf_words = leaf_off, leaf_words
        self.n_int_sym, self.n_leaf_sym = n_int_sym, n_leaf_sym
        self.op_counts = op_counts

    @property
    def n_bricks(self):
        return len(self.n_int_sym)

    def compressed_bytes(self):
        """Bytes of palettes + streams + per-brick header (3 offsets as u64, 2 symbol counts as u32)."""
        n = self.n_bricks
        return 4 * len(self.pal) + 2 * (len(self.int_words) + len(self.leaf_words)) + n * (3 * 8 + 2 * 4)

    def brick_grid(self):
        b = 1 << self.N
        return tuple((d + b - 1) // b for d in self.dims)


def encode_volume(vol, N, stride=1, K_max=32, S_min=256, freq=None, n_threads=None):
    """Encode a volume shaped [Z,Y,X] (x fastest) into a Volume."""
    vol = np.ascontiguousarray(vol, np.uint32)
    Z, Y, X = vol.shape
    rc = C.c_int()
    fp = None
    if freq is not None:
        freq = np.ascontiguousarray(freq, np.uint32)
        fp = _p(freq)
    h = lib().csgvo_encode_volume(_p(vol), _u64x3((X, Y, Z)), N, stride, K_max, S_min, fp,
                                  n_threads or default_threads(), C.byref(rc))
    assert h and rc.value == 0, rc.value
    try:
        sz = np.zeros(4, np.uint64)
        lib().csgvo_volume_sizes(h, sz.ctypes.data_as(C.POINTER(C.c_uint64)))
        n, sp, si, sl = (int(s) for s in sz)
        tabs = np.zeros(32, np.uint32)
        ops = np.zeros(7, np.uint64)
        lib().csgvo_volume_tables(h, _p(tabs), _p(ops))
        pal_off = np.zeros(n + 1, np.uint64)
        int_off = np.zeros(n + 1, np.uint64)
        leaf_off = np.zeros(n + 1, np.uint64)
        pal = np.zeros(max(sp, 1), np.uint32)
        iw = np.zeros(max(si, 1), np.uint16)
        lw = np.zeros(max(sl, 1), np.uint16)
        nis = np.zeros(n, np.uint32)
        nls = np.zeros(n, np.uint32)
        lib().csgvo_volume_export(h, _p(pal_off), _p(pal), _p(int_off), _p(iw), _p(leaf_off), _p(lw), _p(nis),
                                  _p(nls))
        return Volume(N, (X, Y, Z), K_max, S_min, tabs, pal_off, pal[:sp], int_off, iw[:si], leaf_off, lw[:sl],
                      nis, nls, ops)
    finally:
        lib().csgvo_volume_free(h)


def decode_bricks(v: Volume, brick_ids, lods, n_threads=None):
    """Decode requests (brick id, LOD); returns (flat output, offsets, status)."""
    brick_ids = np.ascontiguousarray(brick_ids, np.uint32)
    lods = np.ascontiguousarray(lods, np.uint8)
    n = len(brick_ids)
    sizes = ((1 << v.N) >> lods.astype(np.int64)) ** 3
    out_off = np.zeros(n, np.uint64)
    if n:
        out_off[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(max(int(sizes.sum()), 1), np.uint32)
    status = np.full(n, -1, np.int32)
    pal = v.pal if len(v.pal) else np.zeros(1, np.uint32)
    iw = v.int_words if len(v.int_words) else np.zeros(1, np.uint16)
    lw = v.leaf_words if len(v.leaf_words) else np.zeros(1, np.uint16)
    lib().csgvo_decode_bricks(v.N, v.K_max, v.S_min, _p(v.freq), v.n_bricks, _p(v.pal_off), _p(pal),
                              _p(v.int_off), _p(iw), _p(v.leaf_off), _p(lw), _p(v.n_int_sym), _p(v.n_leaf_sym),
                              _p(brick_ids), _p(lods), n, _p(out), _p(out_off), _p(status),
                              n_threads or default_threads())
    return out, out_off, status
