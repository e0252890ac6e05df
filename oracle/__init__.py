"""CPU oracle for the bitonic sorting library -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The GPU library never does, and
shares no code with it.

Thin ctypes wrappers over ``oracle.c`` (plain C, built with gcc).  Each
function copies its numpy input, so callers' arrays are left untouched.

Functions and the passages they follow:
  bitonic_sort          Section 3.1 network (alternating block directions),
                        with compare-exchange / step / phase counters
                        (Section 3.2 closed forms)
  bitonic_merge         Section 3.1 bitonic merge (half-cleaner steps)
  bitonic_sort_pairs    the same network on (key, original index)
  bitonic_sort_typed    the same network on int32 / float32 / uint64 / int64 /
                        float64 keys (floats: IEEE 754-2008 totalOrder)
  merge_sort[_pairs]    independent stable top-down merge sort
  quicksort             Section 5 / Table 1 CPU comparison (median-of-three)
  std_sort, parallel_sort  std::sort on one core / every core (cpu_baselines.cpp),
                        the benchmark's modern CPU references
  zero_one_failures     0-1 principle over all 2^m zero-one inputs
  segmented_sort[_pairs] per-segment network, ascending
  is_sorted, same_multiset  checkers
"""
from __future__ import annotations

import ctypes
import numpy as np

from . import build as _build


class Counts(ctypes.Structure):
    _fields_ = [("compare_exchanges", ctypes.c_uint64),
                ("steps", ctypes.c_uint64),
                ("phases", ctypes.c_uint64)]


_P32 = ctypes.POINTER(ctypes.c_uint32)
_PI32 = ctypes.POINTER(ctypes.c_int32)
_LIBS: dict[int, ctypes.CDLL] = {}


def load(mutant: int = 0, out_dir: str | None = None) -> ctypes.CDLL:
    key = mutant if out_dir is None else hash((mutant, out_dir))
    if key in _LIBS:
        return _LIBS[key]
    lib = ctypes.CDLL(_build.build(mutant=mutant, out_dir=out_dir))
    u64, i32, i64 = ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
    lib.oracle_bitonic_sort_u32.argtypes = [_P32, u64, i32, i32, ctypes.POINTER(Counts)]
    lib.oracle_bitonic_sort_u32.restype = i32
    lib.oracle_bitonic_merge_u32.argtypes = [_P32, u64, i32, i32]
    lib.oracle_bitonic_merge_u32.restype = i32
    lib.oracle_bitonic_sort_pairs_u32.argtypes = [_P32, _P32, u64, i32, ctypes.POINTER(Counts)]
    lib.oracle_bitonic_sort_pairs_u32.restype = i32
    lib.oracle_segmented_sort_u32.argtypes = [_P32, _PI32, i64]
    lib.oracle_segmented_sort_u32.restype = i32
    lib.oracle_segmented_sort_pairs_u32.argtypes = [_P32, _P32, _PI32, i64]
    lib.oracle_segmented_sort_pairs_u32.restype = i32
    lib.oracle_zero_one_failures.argtypes = [i32, i32, i32]
    lib.oracle_zero_one_failures.restype = u64
    lib.oracle_merge_sort_u32.argtypes = [_P32, u64, i32]
    lib.oracle_merge_sort_u32.restype = i32
    lib.oracle_merge_sort_pairs_u32.argtypes = [_P32, _P32, u64, i32]
    lib.oracle_merge_sort_pairs_u32.restype = i32
    lib.oracle_quicksort_u32.argtypes = [_P32, u64]
    lib.oracle_quicksort_u32.restype = None
    lib.oracle_is_sorted_u32.argtypes = [_P32, u64, i32]
    lib.oracle_is_sorted_u32.restype = i32
    lib.oracle_same_multiset_u32.argtypes = [_P32, _P32, u64]
    lib.oracle_same_multiset_u32.restype = i32
    lib.oracle_bitonic_sort_typed.argtypes = [ctypes.c_void_p, u64, i32, i32, ctypes.POINTER(Counts)]
    lib.oracle_bitonic_sort_typed.restype = i32
    lib.oracle_mutant_id.argtypes = []
    lib.oracle_mutant_id.restype = i32
    _LIBS[key] = lib
    return lib


def _u32(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype.itemsize != 4 or a.dtype.kind not in "iu":
        a = a.astype(np.uint32)
    return np.ascontiguousarray(a).view(np.uint32).copy()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P32)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def bitonic_sort(keys, ascending: bool = True, first_descending: bool = False, lib=None):
    """Section 3.1 network.  Returns (sorted copy, Counts)."""
    lib = lib or load()
    a = _u32(keys)
    c = Counts()
    _check(lib.oracle_bitonic_sort_u32(_ptr(a), a.size, int(ascending), int(first_descending),
                                       ctypes.byref(c)), "bitonic_sort")
    return a, c


# key types of oracle_bitonic_sort_typed
KEY_TYPES = {np.dtype(np.int32): 1, np.dtype(np.float32): 2, np.dtype(np.uint64): 3,
             np.dtype(np.int64): 4, np.dtype(np.float64): 5}


def bitonic_sort_typed(keys, ascending: bool = True, lib=None):
    """Section 3.1 network on int32 / float32 / uint64 / int64 / float64 keys,
    each ordered by its own definition (floats: IEEE 754-2008 totalOrder).
    Returns (sorted copy, Counts); bit patterns are preserved."""
    lib = lib or load()
    a = np.ascontiguousarray(np.asarray(keys)).copy()
    if a.dtype not in KEY_TYPES:
        raise TypeError(f"unsupported key type {a.dtype}")
    c = Counts()
    _check(lib.oracle_bitonic_sort_typed(a.ctypes.data, a.size, KEY_TYPES[a.dtype], int(ascending),
                                         ctypes.byref(c)), "bitonic_sort_typed")
    return a, c


def bitonic_merge(seq, ascending: bool = True, max_steps: int = -1, lib=None):
    lib = lib or load()
    a = _u32(seq)
    _check(lib.oracle_bitonic_merge_u32(_ptr(a), a.size, int(ascending), int(max_steps)),
           "bitonic_merge")
    return a


def bitonic_sort_pairs(keys, vals, ascending: bool = True, lib=None):
    lib = lib or load()
    k, v = _u32(keys), _u32(vals)
    assert k.size == v.size
    c = Counts()
    _check(lib.oracle_bitonic_sort_pairs_u32(_ptr(k), _ptr(v), k.size, int(ascending),
                                             ctypes.byref(c)), "bitonic_sort_pairs")
    return k, v, c


def segmented_sort(keys, offsets, lib=None):
    lib = lib or load()
    k = _u32(keys)
    o = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    _check(lib.oracle_segmented_sort_u32(_ptr(k), o.ctypes.data_as(_PI32), o.size - 1),
           "segmented_sort")
    return k


def segmented_sort_pairs(keys, vals, offsets, lib=None):
    lib = lib or load()
    k, v = _u32(keys), _u32(vals)
    o = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    _check(lib.oracle_segmented_sort_pairs_u32(_ptr(k), _ptr(v), o.ctypes.data_as(_PI32),
                                               o.size - 1), "segmented_sort_pairs")
    return k, v


def zero_one_failures(m: int, ascending: bool = True, first_descending: bool = False, lib=None):
    lib = lib or load()
    return int(lib.oracle_zero_one_failures(int(m), int(ascending), int(first_descending)))


def merge_sort(keys, ascending: bool = True, lib=None):
    lib = lib or load()
    a = _u32(keys)
    _check(lib.oracle_merge_sort_u32(_ptr(a), a.size, int(ascending)), "merge_sort")
    return a


def merge_sort_pairs(keys, vals, ascending: bool = True, lib=None):
    lib = lib or load()
    k, v = _u32(keys), _u32(vals)
    _check(lib.oracle_merge_sort_pairs_u32(_ptr(k), _ptr(v), k.size, int(ascending)),
           "merge_sort_pairs")
    return k, v


def quicksort(keys, lib=None):
    lib = lib or load()
    a = _u32(keys)
    lib.oracle_quicksort_u32(_ptr(a), a.size)
    return a


_CPU_LIB = None


def _cpu_lib() -> ctypes.CDLL:
    """The benchmark's CPU comparison sorts (cpu_baselines.cpp)."""
    global _CPU_LIB
    if _CPU_LIB is None:
        lib = ctypes.CDLL(_build.build_cpu())
        lib.cpu_std_sort_u32.argtypes = [_P32, ctypes.c_uint64]
        lib.cpu_std_sort_u32.restype = None
        lib.cpu_parallel_sort_u32.argtypes = [_P32, ctypes.c_uint64, ctypes.c_int]
        lib.cpu_parallel_sort_u32.restype = ctypes.c_int
        _CPU_LIB = lib
    return _CPU_LIB


def std_sort(keys):
    """std::sort on one core (a modern CPU reference beside Section 5's quicksort)."""
    a = _u32(keys)
    _cpu_lib().cpu_std_sort_u32(_ptr(a), a.size)
    return a


def parallel_sort(keys, threads: int):
    """std::sort of one chunk per thread, then parallel pairwise merges."""
    a = _u32(keys)
    if _cpu_lib().cpu_parallel_sort_u32(_ptr(a), a.size, int(threads)) != 0:
        raise MemoryError("parallel_sort: no scratch buffer")
    return a


def is_sorted(a, ascending: bool = True, lib=None) -> bool:
    lib = lib or load()
    a = _u32(a)
    return bool(lib.oracle_is_sorted_u32(_ptr(a), a.size, int(ascending)))


def same_multiset(a, b, lib=None) -> bool:
    lib = lib or load()
    a, b = _u32(a), _u32(b)
    if a.size != b.size:
        return False
    r = lib.oracle_same_multiset_u32(_ptr(a), _ptr(b), a.size)
    if r < 0:
        raise MemoryError("oracle histogram")
    return bool(r)
