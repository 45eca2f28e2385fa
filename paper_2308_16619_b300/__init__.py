"""Python binding of libcsgv (include/csgv.h): argument marshalling only.

Every step of encoding and decoding runs in the CUDA kernels of libcsgv.so;
this module passes tensor pointers, sizes and the current CUDA stream.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the
library is missing, every call raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcsgv.so")

CSGV_OK, CSGV_PENDING, CSGV_ERR_INVALID_ARG, CSGV_ERR_OOM = 0, 1, 2, 3
CSGV_ERR_CORRUPT, CSGV_ERR_TIMEOUT, CSGV_ERR_CUDA, CSGV_ERR_RANGE = 4, 5, 6, 7

SYMBOLS = ("csgv_last_error", "csgv_build_freq_table", "csgv_encode_bricks", "csgv_decode_bricks",
           "csgv_decode_bricks_plain", "csgv_volume_info_get", "csgv_volume_export", "csgv_volume_import",
           "csgv_volume_destroy", "csgv_encode_bricks_noalloc", "csgv_serve_create", "csgv_serve_submit",
           "csgv_serve_poll", "csgv_serve_release", "csgv_serve_stats_get", "csgv_serve_destroy",
           "csgv_freq_table_from_counts", "csgv_profile_enable", "csgv_profile_reserve", "csgv_profile_read",
           "csgv_decode_autotune", "csgv_decode_get_tuning", "csgv_decode_set_tuning",
           "csgv_volume_leaves_to_host", "csgv_volume_leaves_to_device",
           "csgv_encode_bricks_sampled", "csgv_volume_destroy_async", "csgv_stream_encoder_create",
           "csgv_stream_encoder_add", "csgv_stream_encoder_finish", "csgv_stream_encoder_destroy",
           "csgv_count_bricks", "csgv_footprint_create", "csgv_footprint_frame", "csgv_footprint_destroy")


class CsgvError(RuntimeError):
    pass


class FreqTable(C.Structure):
    _fields_ = [("freq", C.c_uint32 * 32), ("counts", C.c_uint64 * 32)]

    def freq_array(self):
        return np.array(self.freq[:], np.uint32)


class Config(C.Structure):
    _fields_ = [("K_max", C.c_uint32), ("S_min", C.c_uint32)]


class VolumeInfo(C.Structure):
    _fields_ = [("N", C.c_uint32), ("dims", C.c_uint64 * 3), ("grid", C.c_uint64 * 3), ("n_bricks", C.c_uint64),
                ("K_max", C.c_uint32), ("S_min", C.c_uint32), ("max_palette", C.c_uint32),
                ("palette_labels", C.c_uint64), ("int_words", C.c_uint64), ("leaf_words", C.c_uint64),
                ("compressed_bytes", C.c_uint64), ("freq", C.c_uint32 * 32)]


class ServeConfig(C.Structure):
    _fields_ = [("cache_bytes", C.c_uint64), ("max_batch", C.c_uint32), ("n_streams", C.c_uint32)]


class Result(C.Structure):
    _fields_ = [("labels_dev", C.c_void_p), ("status", C.c_int32), ("brick", C.c_uint32), ("lod", C.c_uint8),
                ("pad", C.c_uint8 * 3)]


class DecodeTuning(C.Structure):
    _fields_ = [("workspace_bytes", C.c_uint64), ("rans_ctas_per_sm", C.c_uint32), ("ring_words", C.c_uint32),
                ("rebuild_threads", C.c_uint32), ("medium_threads", C.c_uint32), ("compact_nodes", C.c_uint32),
                ("pad", C.c_uint32), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class Camera(C.Structure):
    """csgv_camera: position, orthonormal basis (right, up, forward) in voxel units, focal length in pixels."""
    _fields_ = [("pos", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3), ("fwd", C.c_float * 3),
                ("f_px", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


class ServeStats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("submitted", "hits", "shared", "misses", "evictions", "rebuilds", "batches",
                                          "decoded_labels", "cache_labels_used", "cache_entries")]


_lib = None


def lib():
    """Load libcsgv.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CsgvError(f"{LIB_PATH} is missing: build it with `python -m paper_2308_16619_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
        L.csgv_decode_autotune.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp, C.POINTER(DecodeTuning)]
        L.csgv_decode_get_tuning.argtypes = [vp, C.POINTER(DecodeTuning)]
        L.csgv_decode_set_tuning.argtypes = [vp, C.POINTER(DecodeTuning)]
        L.csgv_volume_leaves_to_host.argtypes = [vp]
        L.csgv_encode_bricks_sampled.argtypes = [vp, vp, u32, u32, C.POINTER(Config), C.POINTER(FreqTable),
                                                 C.POINTER(vp), vp]
        L.csgv_volume_leaves_to_device.argtypes = [vp]
        L.csgv_profile_enable.argtypes = [C.c_int]
        L.csgv_profile_reserve.argtypes = [u32]
        L.csgv_profile_read.argtypes = [u32, vp, vp, vp, vp]
        L.csgv_last_error.restype = C.c_char_p
        L.csgv_build_freq_table.argtypes = [vp, vp, u32, u32, C.POINTER(FreqTable), vp]
        L.csgv_encode_bricks.argtypes = [vp, vp, u32, C.POINTER(FreqTable), C.POINTER(Config), C.POINTER(vp), vp]
        for f in (L.csgv_decode_bricks, L.csgv_decode_bricks_plain):
            f.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp]
        L.csgv_volume_info_get.argtypes = [vp, C.POINTER(VolumeInfo)]
        L.csgv_volume_export.argtypes = [vp] * 9
        L.csgv_volume_import.argtypes = [u32, vp, u32, u32, vp] + [vp] * 8 + [C.POINTER(vp)]
        L.csgv_volume_destroy.argtypes = [vp]
        L.csgv_volume_destroy.restype = None
        L.csgv_volume_destroy_async.argtypes = [vp, vp]
        L.csgv_stream_encoder_create.argtypes = [vp, u32, C.POINTER(FreqTable), C.POINTER(Config), C.POINTER(vp), vp]
        L.csgv_stream_encoder_add.argtypes = [vp, vp, u64, u32, vp]
        L.csgv_stream_encoder_finish.argtypes = [vp, C.POINTER(vp), vp]
        L.csgv_stream_encoder_destroy.argtypes = [vp]
        L.csgv_stream_encoder_destroy.restype = None
        L.csgv_count_bricks.argtypes = [vp, u32, u32, vp, vp]
        L.csgv_encode_bricks_noalloc.argtypes = [vp, vp, u32, C.POINTER(FreqTable), C.POINTER(Config),
                                                 vp, vp, u64, vp, vp, u64, vp, vp, u64, vp, vp, vp, vp]
        L.csgv_serve_create.argtypes = [vp, C.POINTER(ServeConfig), C.POINTER(vp)]
        L.csgv_serve_submit.argtypes = [vp, vp, vp, u32, C.POINTER(C.c_uint64)]
        L.csgv_serve_poll.argtypes = [vp, u64, u32, C.POINTER(Result)]
        L.csgv_serve_release.argtypes = [vp, u64]
        L.csgv_serve_stats_get.argtypes = [vp, C.POINTER(ServeStats), vp, u32, C.POINTER(C.c_uint32)]
        L.csgv_serve_destroy.argtypes = [vp]
        L.csgv_serve_destroy.restype = None
        L.csgv_freq_table_from_counts.argtypes = [vp, C.POINTER(FreqTable)]
        L.csgv_footprint_create.argtypes = [vp, u32, C.POINTER(vp), vp]
        L.csgv_footprint_frame.argtypes = [vp, C.POINTER(Camera), vp, vp, vp, vp]
        L.csgv_footprint_destroy.argtypes = [vp]
        _lib = L
    return _lib


def _check(rc):
    if rc != CSGV_OK:
        raise CsgvError(f"csgv error {rc}: {lib().csgv_last_error().decode()}")


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def _dims3(vol):
    Z, Y, X = vol.shape
    return (C.c_uint64 * 3)(X, Y, Z)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Volume:
    """A compressed volume held on the device by libcsgv (owns its arrays)."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def info(self):
        inf = VolumeInfo()
        _check(lib().csgv_volume_info_get(self._h, C.byref(inf)))
        return inf

    def export(self):
        """Host copies of the packed arrays (layout as csgv_volume_export)."""
        inf = self.info()
        n = inf.n_bricks
        arrs = dict(pal_off=np.zeros(n + 1, np.uint64), pal=np.zeros(max(inf.palette_labels, 1), np.uint32),
                    int_off=np.zeros(n + 1, np.uint64), int_words=np.zeros(max(inf.int_words, 1), np.uint16),
                    leaf_off=np.zeros(n + 1, np.uint64), leaf_words=np.zeros(max(inf.leaf_words, 1), np.uint16),
                    n_int_sym=np.zeros(n, np.uint32), n_leaf_sym=np.zeros(n, np.uint32))
        order = ("pal_off", "pal", "int_off", "int_words", "leaf_off", "leaf_words", "n_int_sym", "n_leaf_sym")
        _check(lib().csgv_volume_export(self._h, *[arrs[k].ctypes.data_as(C.c_void_p) for k in order]))
        arrs["pal"] = arrs["pal"][:inf.palette_labels]
        arrs["int_words"] = arrs["int_words"][:inf.int_words]
        arrs["leaf_words"] = arrs["leaf_words"][:inf.leaf_words]
        arrs["freq"] = np.array(inf.freq[:], np.uint32)
        return arrs

    def leaves_to_host(self):
        """Detail separation: leaf streams to mapped host memory, read in place by LOD-0 decodes."""
        _check(lib().csgv_volume_leaves_to_host(self._h))

    def leaves_to_device(self):
        _check(lib().csgv_volume_leaves_to_device(self._h))

    def close(self):
        if self._h and self._h.value:
            lib().csgv_volume_destroy(self._h)
            self._h = C.c_void_p(0)

    def close_async(self, stream=None):
        """Free in stream order on `stream` (default: the current stream), without synchronising."""
        if self._h and self._h.value:
            h, self._h = self._h, C.c_void_p(0)
            _check(lib().csgv_volume_destroy_async(h, _stream(stream)))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def csgv_build_freq_table(vol, b, sample_stride=1, stream=None):
    """vol: CUDA tensor [Z, Y, X] of uint32 labels (any 32-bit dtype).  Returns FreqTable."""
    assert vol.is_cuda and vol.element_size() == 4 and vol.is_contiguous()
    t = FreqTable()
    _check(lib().csgv_build_freq_table(_ptr(vol), _dims3(vol), b, sample_stride, C.byref(t), _stream(stream)))
    return t


def csgv_freq_table_from_counts(counts):
    """Tables from 32 nibble counts (interior then leaf), e.g. counts summed over the ranks of a sharded volume."""
    counts = np.ascontiguousarray(counts, np.uint64)
    assert counts.shape == (32,)
    t = FreqTable()
    _check(lib().csgv_freq_table_from_counts(counts.ctypes.data_as(C.c_void_p), C.byref(t)))
    return t


def csgv_encode_bricks(vol, b, table, K_max=32, S_min=256, stream=None):
    assert vol.is_cuda and vol.element_size() == 4 and vol.is_contiguous()
    cfg = Config(K_max, S_min)
    h = C.c_void_p()
    _check(lib().csgv_encode_bricks(_ptr(vol), _dims3(vol), b, C.byref(table), C.byref(cfg), C.byref(h),
                                    _stream(stream)))
    return Volume(h.value)


def csgv_encode_bricks_sampled(vol, b, sample_stride=1, K_max=32, S_min=256, stream=None):
    """Prepass and encode in one call (tables from the nibbles of every sample_stride-th brick of this encode).
    Returns (Volume, FreqTable)."""
    assert vol.is_cuda and vol.element_size() == 4 and vol.is_contiguous()
    cfg = Config(K_max, S_min)
    t = FreqTable()
    h = C.c_void_p()
    _check(lib().csgv_encode_bricks_sampled(_ptr(vol), _dims3(vol), b, sample_stride, C.byref(cfg), C.byref(t),
                                            C.byref(h), _stream(stream)))
    return Volume(h.value), t


def csgv_decode_bricks(volume, brick_ids, lods, out, out_offsets, status, stream=None, plain=False):
    """Device tensors: brick_ids (n, 32-bit), lods (n, uint8), out (32-bit), out_offsets (n, int64), status (n, int32)."""
    n = brick_ids.numel()
    for t in (brick_ids, lods, out, out_offsets, status):
        assert t.is_cuda and t.is_contiguous()
    assert brick_ids.element_size() == 4 and lods.element_size() == 1 and out.element_size() == 4
    assert out_offsets.element_size() == 8 and status.element_size() == 4
    f = lib().csgv_decode_bricks_plain if plain else lib().csgv_decode_bricks
    _check(f(volume.handle, _ptr(brick_ids), _ptr(lods), n, _ptr(out), _ptr(out_offsets), _ptr(status),
             _stream(stream)))


def csgv_decode_autotune(volume, brick_ids, lods, out, out_offsets, status, stream=None):
    """Time decode configurations on this batch, keep the fastest in the volume; returns DecodeTuning."""
    n = brick_ids.numel()
    for t in (brick_ids, lods, out, out_offsets, status):
        assert t.is_cuda and t.is_contiguous()
    best = DecodeTuning()
    _check(lib().csgv_decode_autotune(volume.handle, _ptr(brick_ids), _ptr(lods), n, _ptr(out), _ptr(out_offsets),
                                      _ptr(status), _stream(stream), C.byref(best)))
    return best


def csgv_decode_get_tuning(volume):
    t = DecodeTuning()
    _check(lib().csgv_decode_get_tuning(volume.handle, C.byref(t)))
    return t


def csgv_decode_set_tuning(volume, tuning):
    """Set the volume's decode launch shape (a DecodeTuning); raises on values out of range."""
    _check(lib().csgv_decode_set_tuning(volume.handle, C.byref(tuning)))


def csgv_decode_bricks_plain(volume, brick_ids, lods, out, out_offsets, status, stream=None):
    csgv_decode_bricks(volume, brick_ids, lods, out, out_offsets, status, stream, plain=True)


def csgv_encode_bricks_noalloc(vol, b, table, pal_off, pal, int_off, int_words, leaf_off, leaf_words, n_int_sym,
                               n_leaf_sym, K_max=32, S_min=256, stream=None):
    """Allocation-free encoder, for callers that cannot allocate device memory.

    Writes into the given device tensors (layout of Volume.export) using a fixed scratch array inside
    the library.  Returns (rc, totals): rc is the C status code (0 = OK), totals the numbers of palette
    labels, interior words and leaf words.
    """
    assert vol.is_cuda and vol.element_size() == 4 and vol.is_contiguous()
    # the library cannot see the lengths of the offset and count arrays: check them here, so that a short
    # array is an error and not a device write past its end
    n = 1
    for d in _dims3(vol):
        n *= (d + b - 1) // b
    for name, t, elem, need in (("pal_off", pal_off, 8, n + 1), ("int_off", int_off, 8, n + 1),
                                ("leaf_off", leaf_off, 8, n + 1), ("n_int_sym", n_int_sym, 4, n),
                                ("n_leaf_sym", n_leaf_sym, 4, n), ("pal", pal, 4, 1), ("int_words", int_words, 2, 1),
                                ("leaf_words", leaf_words, 2, 1)):
        if not (t.is_cuda and t.is_contiguous() and t.element_size() == elem):
            raise ValueError(f"{name}: a contiguous CUDA tensor of {elem}-byte elements is needed")
        if t.numel() < need:
            raise ValueError(f"{name}: {t.numel()} elements, {need} needed for {n} bricks")
    cfg = Config(K_max, S_min)
    totals = (C.c_uint64 * 3)()
    rc = lib().csgv_encode_bricks_noalloc(_ptr(vol), _dims3(vol), b, C.byref(table), C.byref(cfg), _ptr(pal_off),
                                          _ptr(pal), pal.numel(), _ptr(int_off), _ptr(int_words), int_words.numel(),
                                          _ptr(leaf_off), _ptr(leaf_words), leaf_words.numel(), _ptr(n_int_sym),
                                          _ptr(n_leaf_sym), totals, _stream(stream))
    return rc, [int(t) for t in totals]


def csgv_volume_import(N, dims_xyz, K_max, S_min, freq, pal_off, pal, int_off, int_words, leaf_off, leaf_words,
                       n_int_sym, n_leaf_sym):
    """Build a device volume from host numpy arrays (layout of Volume.export)."""
    def p(a, dt):
        a = np.ascontiguousarray(a, dt)
        return a, a.ctypes.data_as(C.c_void_p)
    keep = [p(freq, np.uint32), p(pal_off, np.uint64), p(pal if len(pal) else np.zeros(1), np.uint32),
            p(int_off, np.uint64), p(int_words if len(int_words) else np.zeros(1), np.uint16),
            p(leaf_off, np.uint64), p(leaf_words if len(leaf_words) else np.zeros(1), np.uint16),
            p(n_int_sym, np.uint32), p(n_leaf_sym, np.uint32)]
    h = C.c_void_p()
    dims = (C.c_uint64 * 3)(*[int(d) for d in dims_xyz])
    _check(lib().csgv_volume_import(N, dims, K_max, S_min, *[k[1] for k in keep], C.byref(h)))
    return Volume(h.value)


def request_layout(b, lods):
    """Output offsets (int64) for requests decoded back to back: sizes (b >> lod)^3 (host helper for callers)."""
    lods = np.asarray(lods, np.int64)
    sizes = (b >> lods) ** 3
    off = np.zeros(len(lods), np.int64)
    if len(lods):
        off[1:] = np.cumsum(sizes)[:-1]
    return off, int(sizes.sum())


class DeviceView:
    """Zero-copy view of n uint32 labels at a device address (for torch.as_tensor)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<u4", "data": (int(ptr), False),
                                         "version": 3}


class StreamEncoder:
    """Encoder fed with batches of whole bricks in brick-id order (brick-major device tensors of b^3 labels
    per brick); finish() returns the Volume."""

    def __init__(self, dims_xyz, b, table, K_max=32, S_min=256, stream=None):
        self.b = b
        cfg = Config(K_max, S_min)
        h = C.c_void_p()
        dims = (C.c_uint64 * 3)(*dims_xyz)
        _check(lib().csgv_stream_encoder_create(dims, b, C.byref(table), C.byref(cfg), C.byref(h), _stream(stream)))
        self._h = h

    def add(self, bricks, first, stream=None):
        assert bricks.is_cuda and bricks.element_size() == 4 and bricks.is_contiguous()
        m = bricks.numel() // self.b ** 3
        assert m * self.b ** 3 == bricks.numel()
        _check(lib().csgv_stream_encoder_add(self._h, _ptr(bricks), first, m, _stream(stream)))

    def finish(self, stream=None):
        v = C.c_void_p()
        _check(lib().csgv_stream_encoder_finish(self._h, C.byref(v), _stream(stream)))
        self._h = C.c_void_p(0)
        return Volume(v.value)

    def close(self):
        if self._h and self._h.value:
            lib().csgv_stream_encoder_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def csgv_count_bricks(bricks, b, counts=None, stream=None):
    """Add the nibble counts of a brick-major batch to counts (32 uint64, host); returns counts."""
    assert bricks.is_cuda and bricks.element_size() == 4 and bricks.is_contiguous()
    counts = np.zeros(32, np.uint64) if counts is None else counts
    assert counts.dtype == np.uint64 and counts.shape == (32,) and counts.flags.c_contiguous
    _check(lib().csgv_count_bricks(_ptr(bricks), bricks.numel() // b ** 3, b, counts.ctypes.data_as(C.c_void_p),
                                   _stream(stream)))
    return counts


class Server:
    """csgv_serve_*: decode server with a device cache of decoded bricks (see include/csgv.h)."""

    def __init__(self, volume, cache_bytes=0, max_batch=0, n_streams=0):
        self.volume = volume  # keep the volume alive
        h = C.c_void_p()
        cfg = ServeConfig(cache_bytes, max_batch, n_streams)
        _check(lib().csgv_serve_create(volume.handle, C.byref(cfg), C.byref(h)))
        self._h = h
        self.N = volume.info().N

    def submit(self, bricks, lods):
        bricks = np.ascontiguousarray(bricks, np.uint32)
        lods = np.ascontiguousarray(lods, np.uint8)
        t = C.c_uint64()
        _check(lib().csgv_serve_submit(self._h, bricks.ctypes.data_as(C.c_void_p), lods.ctypes.data_as(C.c_void_p),
                                       len(bricks), C.byref(t)))
        return t.value, len(bricks)

    def poll(self, ticket, timeout_us=1_000_000):
        """Returns (rc, results): rc CSGV_OK / CSGV_PENDING / CSGV_ERR_TIMEOUT."""
        tid, n = ticket
        res = (Result * max(n, 1))()
        rc = lib().csgv_serve_poll(self._h, tid, timeout_us, res)
        return rc, (list(res[:n]) if rc == CSGV_OK else None)

    def release(self, ticket):
        _check(lib().csgv_serve_release(self._h, ticket[0]))

    def stats(self, with_latencies=False):
        st = ServeStats()
        cnt = C.c_uint32()
        _check(lib().csgv_serve_stats_get(self._h, C.byref(st), None, 0, C.byref(cnt)))
        lat = None
        if with_latencies:
            lat = np.zeros(max(cnt.value, 1), np.float64)
            _check(lib().csgv_serve_stats_get(self._h, C.byref(st), lat.ctypes.data_as(C.c_void_p), len(lat),
                                              C.byref(cnt)))
            lat = lat[:cnt.value]
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}, lat

    def labels(self, result, b):
        """torch view of a result's labels (valid until the ticket is released)."""
        import torch
        n = (b >> result.lod) ** 3
        return torch.as_tensor(DeviceView(result.labels_dev, n), device="cuda")

    def close(self):
        if self._h and self._h.value:
            lib().csgv_serve_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def profile_enable(on=True):
    """Record CUDA events around every kernel launch of the library (csgv_profile_enable)."""
    _check(lib().csgv_profile_enable(1 if on else 0))


def profile_reserve(n_events):
    """Pre-create n_events timing events for the current device (csgv_profile_reserve): two per timed launch."""
    _check(lib().csgv_profile_reserve(int(n_events)))


def profile_read(max_kernels=32):
    """Per-kernel totals since the last read: {name: (total_ms, launches)} (csgv_profile_read; synchronises)."""
    names = C.create_string_buffer(48 * max_kernels)
    ms = (C.c_double * max_kernels)()
    cnt = (C.c_uint32 * max_kernels)()
    nk = C.c_uint32(0)
    _check(lib().csgv_profile_read(max_kernels, names, ms, cnt, C.byref(nk)))
    out = {}
    for k in range(nk.value):
        nm = names.raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (ms[k], cnt[k])
    return out


def make_camera(pos, right, up, fwd, f_px, width, height):
    """A csgv_camera from three-vectors (rounded to float32)."""
    cam = Camera()
    for name, v in (("pos", pos), ("right", right), ("up", up), ("fwd", fwd)):
        arr = getattr(cam, name)
        for a in range(3):
            arr[a] = float(v[a])
    cam.f_px, cam.width, cam.height = float(f_px), int(width), int(height)
    return cam


class Footprint:
    """csgv_footprint_*: the brick requests of rendered frames (ray walk over the brick grid with empty-space
    skipping; see include/csgv.h).  frame() returns device tensors (bricks int32, lods uint8) of the frame's
    requests in brick-id order."""

    def __init__(self, volume, max_nonempty=1, stream=None):
        import torch
        self.volume = volume  # keep the volume alive
        h = C.c_void_p()
        _check(lib().csgv_footprint_create(volume.handle, max_nonempty, C.byref(h), _stream(stream)))
        self._h = h
        n = volume.info().n_bricks
        self.bricks = torch.empty(n, dtype=torch.int32, device="cuda")
        self.lods = torch.empty(n, dtype=torch.uint8, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int32, device="cuda")

    def frame(self, camera, stream=None):
        _check(lib().csgv_footprint_frame(self._h, C.byref(camera), _ptr(self.bricks), _ptr(self.lods),
                                          _ptr(self.count), _stream(stream)))
        n = int(self.count.item())
        return self.bricks[:n], self.lods[:n]

    def close(self):
        if self._h and self._h.value:
            lib().csgv_footprint_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
