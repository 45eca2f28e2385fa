"""CPU checks of the boundary: libcsgv.so builds for sm_103a, loads, and exports every
entry point include/csgv.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

import paper_2308_16619_b300 as csgv
from paper_2308_16619_b300 import build as csgv_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "csgv.h")).read()
    return sorted(set(re.findall(r"CSGV_API\s+[\w\s\*]*?\b(csgv_\w+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = csgv_build.build()
    lib = ctypes.CDLL(path)
    decl = declared_symbols()
    assert len(decl) >= 9
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(csgv.SYMBOLS) == decl


def test_binding_loads_and_reports_argument_errors_without_gpu():
    L = csgv.lib()
    # argument checks happen on the host before any CUDA call
    t = csgv.FreqTable()
    dims = (ctypes.c_uint64 * 3)(8, 8, 8)
    rc = L.csgv_build_freq_table(None, dims, 8, 1, ctypes.byref(t), None)
    assert rc == csgv.CSGV_ERR_INVALID_ARG
    assert b"NULL" in L.csgv_last_error()
    rc = L.csgv_build_freq_table(ctypes.c_void_p(16), dims, 12, 1, ctypes.byref(t), None)
    assert rc == csgv.CSGV_ERR_INVALID_ARG and b"power of two" in L.csgv_last_error()
    rc = L.csgv_decode_bricks(None, None, None, 0, None, None, None, None)
    assert rc == csgv.CSGV_ERR_INVALID_ARG


def test_sm103a_cubin_only():
    # the library carries sm_103a machine code (checked through the build flags, not by reading the binary)
    assert "arch=compute_103a,code=sm_103a" in " ".join(csgv_build.FLAGS)


def test_table_from_counts_matches_oracle_normalisation():
    # host-only entry point; the oracle's normalisation is an independent implementation of the same rule
    import numpy as np
    import oracle as O
    rng = np.random.default_rng(21)
    for trial in range(300):
        counts = rng.integers(0, 10 ** int(rng.integers(1, 15)), size=32).astype(np.uint64)
        counts[rng.random(32) < 0.3] = 0
        if trial == 0:
            counts[:] = 0
        if trial == 1:
            counts[:] = np.uint64(2 ** 59)  # count * 4080 needs more than 64 bits on both sides
        if trial == 2:
            counts[:16] = 0
            counts[0], counts[5], counts[15] = 2 ** 63, 2 ** 62, 2 ** 62 - 1  # interior total 2^64 - 1
        t = csgv.csgv_freq_table_from_counts(counts)
        want = np.concatenate([O.normalize(counts[:16]), O.normalize(counts[16:])])
        assert list(t.freq) == want.tolist()
        assert list(t.counts) == counts.tolist()


def test_noalloc_encoder_rejects_a_brick_count_that_would_wrap_without_gpu():
    # 2^30 x 2^30 x 16 bricks of 2^3 is 2^64: a 64-bit product wraps to 0; the call must refuse it on the
    # host, before any CUDA call (the pointers are never dereferenced)
    L = csgv.lib()
    t = csgv.FreqTable()
    for i in range(32):
        t.freq[i] = 256
    dims = (ctypes.c_uint64 * 3)(2 ** 31, 2 ** 31, 32)
    totals = (ctypes.c_uint64 * 3)()
    p = ctypes.c_void_p(256)
    rc = L.csgv_encode_bricks_noalloc(p, dims, 2, ctypes.byref(t), None, p, p, 1, p, p, 1, p, p, 1, p, p, totals,
                                      None)
    assert rc == csgv.CSGV_ERR_INVALID_ARG
    msg = L.csgv_last_error()
    assert b"bricks of 2^3" in msg and b"at most" in msg, msg


def test_request_layout_packs_requests_back_to_back():
    import numpy as np
    lods = np.array([0, 5, 1, 5, 2, 0], np.uint8)
    off, total = csgv.request_layout(32, lods)
    sizes = [32768, 1, 4096, 1, 512, 32768]
    assert off.dtype == np.int64 and off.tolist() == [0, 32768, 32769, 36865, 36866, 37378]
    assert total == sum(sizes)
    off0, total0 = csgv.request_layout(16, np.zeros(0, np.uint8))
    assert len(off0) == 0 and total0 == 0
