"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/bitonic.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

import paper_1506_01446_gb300 as bt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.skipif(not os.path.exists(bt.LIB_PATH), reason="CUDA library not built")


def header_symbols():
    src = open(os.path.join(ROOT, "include", "bitonic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bitonic_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = bt.load()
    syms = header_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) <= set(bt.EXPORTS) | set(syms)
    assert set(bt.EXPORTS) == set(syms)


def test_status_strings():
    assert bt.status_string(bt.OK) == "BITONIC_OK"
    assert bt.status_string(bt.ERR_TIMEOUT) == "BITONIC_ERR_TIMEOUT"


def test_argument_errors_need_no_gpu():
    lib = bt.load()
    assert lib.bitonic_sort_u32(None, 10, 1, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_u32(3, 10, 1, None) == bt.ERR_INVALID          # misaligned
    assert lib.bitonic_sort_u32(None, 1, 1, None) == bt.OK                 # n <= 1: nothing to do
    assert lib.bitonic_sort_u32(None, 0, 0, None) == bt.OK
    assert lib.bitonic_sort_u32(16, (1 << 31) + 1, 1, None) == bt.ERR_UNSUPPORTED
    assert lib.bitonic_sort_pairs_u32(16, None, 10, 1, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_segmented_u32(16, None, 4, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_segmented_u32(16, 16, -1, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_segmented_u32(16, 16, 0, None) == bt.OK
    assert lib.bitonic_sort_segmented_pairs_u32(16, None, 16, 3, None) == bt.ERR_INVALID
    for asc in (1, 0):  # either direction checks every argument before any launch
        assert lib.bitonic_sort_segmented_u32_dir(16, None, 4, asc, None) == bt.ERR_INVALID
        assert lib.bitonic_sort_segmented_u32_dir(16, 16, -1, asc, None) == bt.ERR_INVALID
        assert lib.bitonic_sort_segmented_u32_dir(16, 16, 0, asc, None) == bt.OK
        assert lib.bitonic_sort_segmented_u32_dir(3, 16, 4, asc, None) == bt.ERR_INVALID    # misaligned keys
        assert lib.bitonic_sort_segmented_u32_dir(16, 18, 4, asc, None) == bt.ERR_INVALID   # misaligned offsets
        assert lib.bitonic_sort_segmented_pairs_u32_dir(16, None, 16, 3, asc, None) == bt.ERR_INVALID
        assert lib.bitonic_sort_segmented_pairs_u32_dir(16, 18, 16, 3, asc, None) == bt.ERR_INVALID
        assert lib.bitonic_sort_segmented_pairs_u32_dir(16, 16, 16, 0, asc, None) == bt.OK
    assert lib.bitonic_sort_u32_profiled(16, 100, 1, None, None, 0, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_u32_host(None, None, 0, 1, None) == bt.OK
    assert lib.bitonic_sort_u32_host(None, 16, 10, 1, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_u32_host(16, None, 10, 1, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_u32_host(16, 16, (1 << 31) + 1, 1, None) == bt.ERR_UNSUPPORTED
    assert lib.bitonic_sort_u32_host_batch(None, None, None, 0, 1, None) == bt.OK
    assert lib.bitonic_sort_u32_host_batch(None, None, None, -1, 1, None) == bt.ERR_INVALID
    assert lib.bitonic_sort_u32_host_batch(None, None, None, 2, 1, None) == bt.ERR_INVALID
    ptrs = (ctypes.c_void_p * 2)(16, None)
    ns = (ctypes.c_size_t * 2)(10, 10)
    assert lib.bitonic_sort_u32_host_batch(ptrs, ptrs, ns, 2, 1, None) == bt.ERR_INVALID
    for name, size in (("bitonic_sort_i32", 4), ("bitonic_sort_f32", 4), ("bitonic_sort_u64", 8),
                       ("bitonic_sort_i64", 8), ("bitonic_sort_f64", 8)):
        f = getattr(lib, name)
        assert f(None, 10, 1, None) == bt.ERR_INVALID, name
        assert f(size // 2, 10, 1, None) == bt.ERR_INVALID, name        # not aligned to the key size
        assert f(None, 1, 0, None) == bt.OK, name
        assert f(16, (1 << 31) + 1, 1, None) == bt.ERR_UNSUPPORTED, name


def test_options_validation():
    saved = bt.get_options()
    try:
        with pytest.raises(bt.BitonicError):
            bt.set_options(variant=7)
        with pytest.raises(bt.BitonicError):
            bt.set_options(tile_log2=20)
        bt.set_options(variant=2, tile_log2=13)
        assert bt.get_options()["variant"] == 2
    finally:
        bt.set_options(**saved)


def test_thread_graph_mode_validation():
    lib = bt.load()
    for mode in (-1, 0, 1):
        assert lib.bitonic_set_thread_graphs(mode) == bt.OK
    for mode in (-2, 2, 7):
        assert lib.bitonic_set_thread_graphs(mode) == bt.ERR_INVALID
    with bt.thread_graphs(False):
        pass
    assert lib.bitonic_set_thread_graphs(-1) == bt.OK


def test_debug_wait_argument_check_needs_no_gpu():
    # a starving test mode needs a bound of at least one try (checked before
    # any device work)
    assert bt.load().bitonic_debug_set_wait(1, 0) == bt.ERR_INVALID


def test_serve_run_rejects_bad_arguments_before_any_cuda_call():
    import numpy as np
    lib = bt.load()
    dt = bt.serve_request_dtype()
    assert dt.itemsize == 24
    stats = bt.ServeStats()
    done = np.zeros(4, dtype=np.float64)
    pos = np.zeros(4, dtype=np.uint64)
    streams = (ctypes.c_void_p * 1)(None)

    def cfg(**kw):
        base = dict(dev_arena=4096, dev_bytes=1 << 20, in_keys=4096, in_vals=4096, pool_len=1 << 16,
                    out_keys=4096, out_vals=4096, out_cap=1 << 16, offs_stage=4096, offs_cap=1024,
                    streams=streams, nstreams=1, small_keys=16384, small_pairs=8192, max_batch=64, keep_outputs=0)
        base.update(kw)
        return bt.ServeConfig(**base)

    def run(c, reqs):
        r = np.zeros(len(reqs), dtype=dt)
        for i, (a, src, n, hv) in enumerate(reqs):
            r[i] = (a, src, n, hv)
        return lib.bitonic_serve_run(ctypes.byref(c) if c is not None else None, r.ctypes.data, len(reqs),
                                     done.ctypes.data, pos.ctypes.data, ctypes.byref(stats))

    assert run(None, []) == bt.ERR_INVALID
    assert run(cfg(), []) == bt.OK                                            # nothing to serve
    assert run(cfg(dev_arena=4100), [(0.0, 0, 10, 0)]) == bt.ERR_INVALID      # arena not 16-byte aligned
    assert run(cfg(nstreams=0), [(0.0, 0, 10, 0)]) == bt.ERR_INVALID
    assert run(cfg(small_keys=1 << 15), [(0.0, 0, 10, 0)]) == bt.ERR_INVALID  # beyond one packed tile
    assert run(cfg(), [(0.0, 0, 0, 0)]) == bt.ERR_INVALID                     # empty request
    assert run(cfg(), [(0.0, (1 << 16) - 5, 10, 0)]) == bt.ERR_INVALID        # source beyond the pool
    assert run(cfg(), [(1.0, 0, 10, 0), (0.5, 0, 10, 0)]) == bt.ERR_INVALID   # arrivals out of order
    assert run(cfg(in_vals=None), [(0.0, 0, 10, 1)]) == bt.ERR_INVALID        # values without a pool
    assert run(cfg(dev_bytes=1 << 12), [(0.0, 0, 5000, 0)]) == bt.ERR_INVALID  # never fits the arena
    assert run(cfg(out_cap=100), [(0.0, 0, 200, 0)]) == bt.ERR_INVALID        # never fits the output area
    assert run(cfg(keep_outputs=1, out_cap=300), [(0.0, 0, 200, 0), (0.0, 200, 200, 0)]) == bt.ERR_INVALID
    assert "keep_outputs" in bt.last_error_message()
