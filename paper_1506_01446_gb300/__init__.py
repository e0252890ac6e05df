"""GB300 (sm_103a) bitonic sorting library -- Python binding.

Thin ctypes shims over the C ABI declared in ``include/bitonic.h``: argument
marshalling only, every step of a sort runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the
CUDA library is missing, :func:`load` raises.

The sort is Batcher's bitonic network as described by Mu, Cui and Song,
"The implementation and optimization of Bitonic sort algorithm based on CUDA"
(Section 3.1 network, Section 3.3 one kernel per step, Section 4.1 shared
memory, Section 4.2 registers).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libbitonic.so")

OK, ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)
VARIANT_OPTIMIZED, VARIANT_BASIC, VARIANT_SEMI = 0, 1, 2
KIND_NAMES = {0: "tile_sort", 1: "global_pass", 2: "tile_merge", 3: "step"}

# Every symbol include/bitonic.h declares.
EXPORTS = (
    "bitonic_sort_u32", "bitonic_sort_pairs_u32", "bitonic_sort_segmented_u32",
    "bitonic_sort_segmented_pairs_u32", "bitonic_status_string", "bitonic_last_error_message",
    "bitonic_last_device_error", "bitonic_release_workspace", "bitonic_set_options",
    "bitonic_get_options", "bitonic_plan_info", "bitonic_sort_u32_profiled", "bitonic_debug_plan",
    "bitonic_debug_desc_size", "bitonic_sort_pairs_u32_noalloc", "bitonic_sort_segmented_pairs_u32_bounded",
    "bitonic_set_class_options", "bitonic_sort_i32", "bitonic_sort_f32", "bitonic_sort_u64", "bitonic_sort_i64",
    "bitonic_sort_f64", "bitonic_sort_u32_host", "bitonic_sort_u32_host_batch",
    "bitonic_sort_segmented_u32_dir", "bitonic_sort_segmented_pairs_u32_dir", "bitonic_set_thread_graphs",
    "bitonic_debug_set_wait", "bitonic_set_segmented_options", "bitonic_serve_run", "bitonic_graph_kernels",
)

# torch dtype name -> C entry point of the keys-only sorts (uint64 keys may be
# held in an int64 tensor: pass key_type="uint64")
KEY_TYPE_ENTRY = {"int32": "bitonic_sort_i32", "float32": "bitonic_sort_f32", "uint64": "bitonic_sort_u64",
                  "int64": "bitonic_sort_i64", "float64": "bitonic_sort_f64", "uint32": "bitonic_sort_u32"}


class BitonicError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} {last_error_message()}".rstrip())


class Options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("tile_log2", ctypes.c_int),
                ("global_bits", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("keys_per_thread_log2", ctypes.c_int), ("io_direct", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("min_row_log2", ctypes.c_int), ("l2_prefetch", ctypes.c_int),
                ("pipeline", ctypes.c_int), ("round_sync", ctypes.c_int), ("split_log2", ctypes.c_int)]


class SegOptions(ctypes.Structure):
    _fields_ = [("tile_log2", ctypes.c_int), ("class_floor_gap", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


class ServeConfig(ctypes.Structure):
    """bitonic_serve_config (include/bitonic.h)."""
    _fields_ = [("dev_arena", ctypes.c_void_p), ("dev_bytes", ctypes.c_size_t),
                ("in_keys", ctypes.c_void_p), ("in_vals", ctypes.c_void_p), ("pool_len", ctypes.c_size_t),
                ("out_keys", ctypes.c_void_p), ("out_vals", ctypes.c_void_p), ("out_cap", ctypes.c_size_t),
                ("offs_stage", ctypes.c_void_p), ("offs_cap", ctypes.c_size_t),
                ("streams", ctypes.POINTER(ctypes.c_void_p)), ("nstreams", ctypes.c_int),
                ("small_keys", ctypes.c_uint32), ("small_pairs", ctypes.c_uint32), ("max_batch", ctypes.c_int),
                ("keep_outputs", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    """bitonic_serve_stats (include/bitonic.h)."""
    _fields_ = [("span_s", ctypes.c_double), ("batches", ctypes.c_int64), ("batched_requests", ctypes.c_int64),
                ("large_launches", ctypes.c_int64), ("peak_device_bytes", ctypes.c_uint64)]


def serve_request_dtype():
    """numpy layout of bitonic_serve_request."""
    import numpy as np
    return np.dtype([("arrival_s", "<f8"), ("src", "<u8"), ("n", "<u4"), ("has_vals", "<i4")])


_lib = None


def load() -> ctypes.CDLL:
    """Loads libbitonic.so (built by ``paper_1506_01446_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    pint = ctypes.POINTER(ctypes.c_int)
    lib.bitonic_sort_u32.argtypes = [vp, sz, i32, vp]
    for name in ("bitonic_sort_i32", "bitonic_sort_f32", "bitonic_sort_u64", "bitonic_sort_i64", "bitonic_sort_f64"):
        getattr(lib, name).argtypes = [vp, sz, i32, vp]
    lib.bitonic_sort_u32_host.argtypes = [vp, vp, sz, i32, vp]
    lib.bitonic_sort_u32_host_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(sz), i32,
                                                i32, vp]
    lib.bitonic_sort_pairs_u32.argtypes = [vp, vp, sz, i32, vp]
    lib.bitonic_sort_segmented_u32.argtypes = [vp, vp, i32, vp]
    lib.bitonic_sort_segmented_pairs_u32.argtypes = [vp, vp, vp, i32, vp]
    lib.bitonic_sort_segmented_u32_dir.argtypes = [vp, vp, i32, i32, vp]
    lib.bitonic_sort_segmented_pairs_u32_dir.argtypes = [vp, vp, vp, i32, i32, vp]
    lib.bitonic_status_string.argtypes = [i32]
    lib.bitonic_status_string.restype = ctypes.c_char_p
    lib.bitonic_last_error_message.argtypes = []
    lib.bitonic_last_error_message.restype = ctypes.c_char_p
    lib.bitonic_last_device_error.argtypes = [vp]
    lib.bitonic_release_workspace.argtypes = []
    lib.bitonic_set_options.argtypes = [ctypes.POINTER(Options)]
    lib.bitonic_get_options.argtypes = [ctypes.POINTER(Options)]
    lib.bitonic_plan_info.argtypes = [sz, i32, pint, pint, pint, pint]
    lib.bitonic_graph_kernels.argtypes = [sz, i32, pint]
    lib.bitonic_sort_u32_profiled.argtypes = [vp, sz, i32, vp, ctypes.POINTER(vp), i32, pint]
    lib.bitonic_debug_plan.argtypes = [sz, i32, pint, i32, vp, i32]
    lib.bitonic_debug_desc_size.argtypes = []
    lib.bitonic_debug_desc_size.restype = sz
    lib.bitonic_sort_pairs_u32_noalloc.argtypes = [vp, vp, sz, i32, vp]
    lib.bitonic_sort_segmented_pairs_u32_bounded.argtypes = [vp, vp, vp, i32, i32, vp]
    lib.bitonic_set_class_options.argtypes = [i32, i32, ctypes.POINTER(Options)]
    lib.bitonic_set_thread_graphs.argtypes = [i32]
    lib.bitonic_debug_set_wait.argtypes = [i32, ctypes.c_uint]
    lib.bitonic_set_segmented_options.argtypes = [i32, i32, ctypes.POINTER(SegOptions)]
    lib.bitonic_serve_run.argtypes = [ctypes.POINTER(ServeConfig), vp, i32, vp, vp, ctypes.POINTER(ServeStats)]
    for name in EXPORTS:
        f = getattr(lib, name)
        if f.restype is ctypes.c_int or f.restype is None:
            pass
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().bitonic_status_string(int(status)).decode()


def last_error_message() -> str:
    return load().bitonic_last_error_message().decode()


def _check(status: int, what: str):
    if status != OK:
        raise BitonicError(status, what)


def _stream_handle(stream):
    """cudaStream_t of a torch stream (None = torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _u32_ptr(t, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.element_size() != 4:
        raise ValueError(f"{name} must have 4-byte elements (uint32 or int32 view)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def sort_(keys, ascending: bool = True, stream=None):
    """Sorts a CUDA tensor of 32-bit keys in place (unsigned order)."""
    _check(load().bitonic_sort_u32(_u32_ptr(keys, "keys"), keys.numel(), int(bool(ascending)),
                                   _stream_handle(stream)), "bitonic_sort_u32")
    return keys


def sort_typed_(keys, ascending: bool = True, stream=None, key_type: str | None = None):
    """Sorts a CUDA tensor in place by its element type's order: int32,
    float32, int64, float64 (floats: IEEE 754 totalOrder), uint32 / uint64
    (key_type "uint32" for an int32 tensor holding unsigned keys, "uint64"
    for an int64 tensor)."""
    if not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA tensor")
    kt = key_type or str(keys.dtype).replace("torch.", "")
    entry = KEY_TYPE_ENTRY.get(kt)
    if entry is None:
        raise ValueError(f"unsupported key type {kt}")
    if keys.element_size() != (8 if kt in ("uint64", "int64", "float64") else 4):
        raise ValueError(f"{kt} keys need {8 if '64' in kt else 4}-byte elements")
    _check(getattr(load(), entry)(keys.data_ptr(), keys.numel(), int(bool(ascending)), _stream_handle(stream)),
           entry)
    return keys


def sort_host(keys_in, keys_out=None, ascending: bool = True, stream=None):
    """Sorts 32-bit keys held in HOST memory (CPU tensors; page-locked for
    asynchronous copies) into keys_out (default: in place).  Work is
    enqueued on the CUDA stream; synchronise before reading keys_out."""
    if keys_out is None:
        keys_out = keys_in
    for t, name in ((keys_in, "keys_in"), (keys_out, "keys_out")):
        if t.is_cuda or t.element_size() != 4 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor of 4-byte keys")
    if keys_in.numel() != keys_out.numel():
        raise ValueError("keys_in and keys_out differ in length")
    _check(load().bitonic_sort_u32_host(keys_in.data_ptr(), keys_out.data_ptr(), keys_in.numel(),
                                        int(bool(ascending)), _stream_handle(stream)), "bitonic_sort_u32_host")
    return keys_out


def sort_host_batch(keys_in, keys_out=None, ascending: bool = True, stream=None):
    """Sorts a list of host tensors of 32-bit keys (page-locked for
    asynchronous copies) into keys_out (default: in place), overlapping each
    array's copies with its neighbours' passes.  Synchronise the stream
    before reading keys_out."""
    if keys_out is None:
        keys_out = keys_in
    if len(keys_in) != len(keys_out):
        raise ValueError("keys_in and keys_out differ in length")
    for a, b in zip(keys_in, keys_out):
        for t in (a, b):
            if t.is_cuda or t.element_size() != 4 or not t.is_contiguous():
                raise ValueError("every array must be a contiguous host tensor of 4-byte keys")
        if a.numel() != b.numel():
            raise ValueError("an input and its output differ in length")
    k = len(keys_in)
    ins = (ctypes.c_void_p * k)(*[t.data_ptr() for t in keys_in])
    outs = (ctypes.c_void_p * k)(*[t.data_ptr() for t in keys_out])
    ns = (ctypes.c_size_t * k)(*[t.numel() for t in keys_in])
    _check(load().bitonic_sort_u32_host_batch(ins, outs, ns, k, int(bool(ascending)), _stream_handle(stream)),
           "bitonic_sort_u32_host_batch")
    return keys_out


def sort_pairs_(keys, vals, ascending: bool = True, stream=None):
    """Sorts key/value pairs in place; equal keys keep their original order."""
    if keys.numel() != vals.numel():
        raise ValueError("keys and vals differ in length")
    _check(load().bitonic_sort_pairs_u32(_u32_ptr(keys, "keys"), _u32_ptr(vals, "vals"), keys.numel(),
                                         int(bool(ascending)), _stream_handle(stream)),
           "bitonic_sort_pairs_u32")
    return keys, vals


def _offsets_ptr(offsets):
    import torch
    if not offsets.is_cuda or offsets.dtype != torch.int32 or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous int32 CUDA tensor")
    return offsets.data_ptr()


def sort_segmented_(keys, offsets, stream=None, ascending: bool = True):
    """Sorts keys[offsets[s]:offsets[s+1]] for every segment s (ascending, or
    descending through bitonic_sort_segmented_u32_dir)."""
    nseg = offsets.numel() - 1
    if ascending:
        _check(load().bitonic_sort_segmented_u32(_u32_ptr(keys, "keys"), _offsets_ptr(offsets), nseg,
                                                 _stream_handle(stream)), "bitonic_sort_segmented_u32")
    else:
        _check(load().bitonic_sort_segmented_u32_dir(_u32_ptr(keys, "keys"), _offsets_ptr(offsets), nseg, 0,
                                                     _stream_handle(stream)), "bitonic_sort_segmented_u32_dir")
    return keys


def sort_segmented_pairs_(keys, vals, offsets, stream=None, ascending: bool = True):
    nseg = offsets.numel() - 1
    if ascending:
        _check(load().bitonic_sort_segmented_pairs_u32(_u32_ptr(keys, "keys"), _u32_ptr(vals, "vals"),
                                                       _offsets_ptr(offsets), nseg, _stream_handle(stream)),
               "bitonic_sort_segmented_pairs_u32")
    else:
        _check(load().bitonic_sort_segmented_pairs_u32_dir(_u32_ptr(keys, "keys"), _u32_ptr(vals, "vals"),
                                                           _offsets_ptr(offsets), nseg, 0, _stream_handle(stream)),
               "bitonic_sort_segmented_pairs_u32_dir")
    return keys, vals


def sort_segmented_pairs_bounded_(keys, vals, offsets, max_len: int, stream=None):
    """Segmented pair sort for segments known to be at most max_len long
    (fully asynchronous when max_len <= 8192)."""
    nseg = offsets.numel() - 1
    _check(load().bitonic_sort_segmented_pairs_u32_bounded(_u32_ptr(keys, "keys"), _u32_ptr(vals, "vals"),
                                                           _offsets_ptr(offsets), nseg, int(max_len),
                                                           _stream_handle(stream)),
           "bitonic_sort_segmented_pairs_u32_bounded")
    return keys, vals


def last_device_error(stream=None) -> int:
    """Synchronises the stream and returns (and clears) its device status."""
    return load().bitonic_last_device_error(_stream_handle(stream))


def release_workspace():
    _check(load().bitonic_release_workspace(), "bitonic_release_workspace")


def get_options() -> dict:
    o = Options()
    _check(load().bitonic_get_options(ctypes.byref(o)), "bitonic_get_options")
    return {f: getattr(o, f) for f, _ in Options._fields_}


def set_options(variant=None, tile_log2=None, global_bits=None, use_graph=None,
                keys_per_thread_log2=None, io_direct=None, pipeline=None, l2_prefetch=None,
                min_row_log2=None, ctas_per_sm=None, round_sync=None, split_log2=None):
    cur = get_options()
    for k, v in (("variant", variant), ("tile_log2", tile_log2), ("global_bits", global_bits),
                 ("use_graph", use_graph), ("keys_per_thread_log2", keys_per_thread_log2),
                 ("io_direct", io_direct), ("pipeline", pipeline), ("l2_prefetch", l2_prefetch),
                 ("min_row_log2", min_row_log2), ("ctas_per_sm", ctas_per_sm), ("round_sync", round_sync),
                 ("split_log2", split_log2)):
        if v is not None:
            cur[k] = int(v)
    _check(load().bitonic_set_options(ctypes.byref(Options(**cur))), "bitonic_set_options")
    return cur


def debug_set_wait(starve_copies: bool, max_spins: int = 0):
    """Testing aid: the pipelined kernels' copy-starving mode with a short
    wait bound (their waits then time out), or normal operation."""
    _check(load().bitonic_debug_set_wait(int(bool(starve_copies)), int(max_spins)), "bitonic_debug_set_wait")


class thread_graphs:
    """Context manager: graph replay on (True), off (False) or following the
    process-wide option (None) for the library calls of this host thread."""

    def __init__(self, enabled):
        self.mode = -1 if enabled is None else int(bool(enabled))

    def __enter__(self):
        _check(load().bitonic_set_thread_graphs(self.mode), "bitonic_set_thread_graphs")
        return self

    def __exit__(self, *exc):
        load().bitonic_set_thread_graphs(-1)
        return False


def set_segmented_options(pairs: bool, log2_nseg: int, options: dict | None):
    """Installs (or with None removes) the packed-tile choice of segmented
    sorts of 2^(log2_nseg - 1) < nseg <= 2^log2_nseg segments."""
    ptr = None
    if options is not None:
        ptr = ctypes.byref(SegOptions(**{**{f: 0 for f, _ in SegOptions._fields_}, **options}))
    _check(load().bitonic_set_segmented_options(int(bool(pairs)), int(log2_nseg), ptr),
           "bitonic_set_segmented_options")


def set_class_options(key_bytes: int, log2_n: int, options: dict | None):
    """Installs (or with None removes) the tuned options of one size class."""
    ptr = None
    if options is not None:
        o = Options(**{**{f: 0 for f, _ in Options._fields_}, **options})
        ptr = ctypes.byref(o)
    _check(load().bitonic_set_class_options(int(key_bytes), int(log2_n), ptr), "bitonic_set_class_options")


def plan_info(n: int, pairs: bool = False) -> dict:
    out = [ctypes.c_int() for _ in range(4)]
    _check(load().bitonic_plan_info(int(n), int(bool(pairs)), *[ctypes.byref(x) for x in out]),
           "bitonic_plan_info")
    return dict(zip(("launches", "hbm_passes", "fused_steps", "global_steps"), (x.value for x in out)))


def graph_kernels(n: int, pairs: bool = False) -> int:
    """Kernels one graph-replayed sort of n keys launches (bitonic_graph_kernels)."""
    out = ctypes.c_int()
    _check(load().bitonic_graph_kernels(int(n), int(bool(pairs)), ctypes.byref(out)), "bitonic_graph_kernels")
    return out.value


def desc_dtype():
    """numpy layout of one launch descriptor (TileParamsBig in csrc/desc.h)."""
    import numpy as np
    rnd = np.dtype([("thr_loc", "<u2", 10), ("reg_loc", "<u2", 5), ("nsteps", "u1"),
                    ("steps", "u1", 36), ("pattern", "u1"), ("warp_local", "u1"), ("pad_r", "u1"),
                    ("thr_sw", "<u2", 10), ("reg_sw", "<u2", 5)])
    io = np.dtype([("thr_glob", "<u4", 10), ("reg_glob", "<u4", 5)])
    return np.dtype([("gvec", "<u4", 16), ("io", io, 2), ("span_mask", "<u4"), ("run_shift", "u1", 4),
                     ("run_width", "u1", 4), ("m", "u1"), ("nruns", "u1"), ("contiguous", "u1"),
                     ("nrounds", "u1"), ("row_log", "u1"), ("pad2", "u1", 3), ("rounds", rnd, 100)])


def debug_plan(n: int, key_bytes: int = 4) -> dict:
    """The launch plan the library builds for a sort of n keys of key_bytes
    bytes under the current options (host code only, no GPU): the tile
    configuration, per launch (kind, phase, hi, lo, flip, descriptor, grid),
    and the descriptors."""
    import numpy as np
    lib = load()
    dt = desc_dtype()
    if lib.bitonic_debug_desc_size() != dt.itemsize:
        raise RuntimeError("descriptor layout does not match the library")
    info = (ctypes.c_int * (6 + 7 * 4096))()
    descs = np.zeros(256, dtype=dt)
    _check(lib.bitonic_debug_plan(int(n), int(key_bytes), info, len(info), descs.ctypes.data, len(descs)),
           "bitonic_debug_plan")
    N, cfg, log_r, log_t, L, D = info[:6]
    launches = [tuple(info[6 + 7 * i: 13 + 7 * i]) for i in range(L)]
    return dict(N=N, cfg=cfg, log_r=log_r, log_t=log_t, launches=launches, descs=descs[:D])


def round_shapes(plan: dict) -> list:
    """Per launch of a debug_plan, the number of network steps in each of its
    register rounds (rounds are joined by a shared-memory transpose; a round
    without steps only changes the layout for coalesced global access)."""
    out = []
    for la in plan["launches"]:
        d = plan["descs"][la[5]]
        out.append(tuple(int(d["rounds"][r]["nsteps"]) for r in range(int(d["nrounds"]))))
    return out


def sort_profiled_(keys, events, ascending: bool = True, stream=None):
    """Like sort_ but without a graph, recording events[i] before launch i and
    events[L] after the last; returns the kernel kind of each launch."""
    n_ev = len(events)
    for e in events:
        if not e.cuda_event:  # torch creates the CUDA event on first record
            e.record()
    arr = (ctypes.c_void_p * n_ev)(*[e.cuda_event for e in events])
    kinds = (ctypes.c_int * n_ev)()
    _check(load().bitonic_sort_u32_profiled(_u32_ptr(keys, "keys"), keys.numel(), int(bool(ascending)),
                                            _stream_handle(stream), arr, n_ev, kinds),
           "bitonic_sort_u32_profiled")
    return list(kinds)
