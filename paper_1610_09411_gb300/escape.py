"""Thin Python binding of the C ABI in include/escape.h (argument marshalling only).

Every function has the name of the C entry point it wraps.  Host inputs are
numpy arrays; device inputs are torch CUDA tensors (their data pointers are
passed with ESCAPE_DEVICE_PTRS).  Streams default to torch's current stream
when torch has initialised CUDA, else the legacy default stream.

There is no fallback: if the compiled library is missing, importing this
module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ESCAPE_HOST_PTRS = 0
ESCAPE_DEVICE_PTRS = 1
ESCAPE_NORMALIZE = 2
ESCAPE_PART_PUT = 4
ESCAPE_PART_SUMS = 64

STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EOVERFLOW", 5: "ETIMEOUT", 6: "EINTERNAL"}
N_PHASES = 9
PHASE_NAMES = ["orient", "triangles", "cliques", "cycles4", "tri_lists", "pairs", "wheels", "cycles5", "assemble"]


class EscapeError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


class U128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]


class Census(ctypes.Structure):
    _fields_ = [("c3", U128 * 4), ("c4", U128 * 11), ("c5", U128 * 34),
                ("n3", U128 * 4), ("n4", U128 * 11), ("n5", U128 * 34)]

    def to_dict(self) -> dict:
        def ints(arr):
            return [int(x.lo) | (int(x.hi) << 64) for x in arr]
        return {k: ints(getattr(self, k)) for k in ("c3", "c4", "c5", "n3", "n4", "n5")}


class Census4(ctypes.Structure):
    _fields_ = [("c3", U128 * 4), ("c4", U128 * 11), ("n3", U128 * 4), ("n4", U128 * 11)]

    def to_dict(self) -> dict:
        def ints(arr):
            return [int(x.lo) | (int(x.hi) << 64) for x in arr]
        return {k: ints(getattr(self, k)) for k in ("c3", "c4", "n3", "n4")}


def _load():
    lib_path = _build.LIB
    if not os.path.exists(lib_path):
        raise ImportError(f"CUDA library not built: {lib_path} (run paper_1610_09411_gb300.build)")
    lib = ctypes.CDLL(lib_path)
    P, i64, u32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
    lib.escape_load_csr.restype = c_int
    lib.escape_load_csr.argtypes = [i64, i64, P, P, u32, P, ctypes.POINTER(P)]
    lib.escape_graph_info.restype = c_int
    lib.escape_graph_info.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.escape_census4.restype = c_int
    lib.escape_census4.argtypes = [P, ctypes.POINTER(Census4), P]
    lib.escape_census5.restype = c_int
    lib.escape_census5.argtypes = [P, ctypes.POINTER(Census), P]
    lib.escape_census5_batch.restype = c_int
    lib.escape_census5_batch.argtypes = [ctypes.c_int32, P, P, P, u32, P, P]
    lib.escape_per_element.restype = c_int
    lib.escape_per_element.argtypes = [P, P, P, P, P, P, P, P]
    lib.escape_set_options.restype = c_int
    lib.escape_set_options.argtypes = [P, c_int, c_int, c_int]
    lib.escape_last_phase_ms.restype = c_int
    lib.escape_last_phase_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float), c_int]
    lib.escape_last_kernel_launches.restype = ctypes.c_longlong
    lib.escape_last_kernel_launches.argtypes = [P]
    lib.escape_census5_part.restype = c_int
    lib.escape_census5_part.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P]
    lib.escape_part_counts.restype = c_int
    lib.escape_part_counts.argtypes = [P, P, P, P, u32, P]
    lib.escape_census5_finish.restype = c_int
    lib.escape_census5_finish.argtypes = [P, P, ctypes.POINTER(Census), P]
    lib.escape_part_sum_count.restype = c_int
    lib.escape_part_sum_count.argtypes = []
    lib.escape_last_basis_counts.restype = c_int
    lib.escape_last_basis_counts.argtypes = [P, P]
    lib.escape_cycles4_noalloc.restype = c_int
    lib.escape_cycles4_noalloc.argtypes = [i64, P, P, P, P, P]
    lib.escape_free.restype = None
    lib.escape_free.argtypes = [P]
    lib.escape_status_str.restype = ctypes.c_char_p
    lib.escape_status_str.argtypes = [c_int]
    lib.escape_last_cuda_error.restype = c_int
    lib.escape_last_cuda_error.argtypes = [ctypes.POINTER(ctypes.c_char_p)]
    return lib


LIB = _load()


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def escape_last_cuda_error():
    """(code, name) of the last CUDA error the library turned into a status
    on this thread; (0, "") if none."""
    name = ctypes.c_char_p()
    code = LIB.escape_last_cuda_error(ctypes.byref(name))
    return code, (name.value or b"").decode()


def _check(code: int, what: str):
    if code != 0:
        if code == 3:                  # ECUDA: name the CUDA error behind it
            cu, name = escape_last_cuda_error()
            if cu:
                what = f"{what} [{name} ({cu})]"
        raise EscapeError(code, what)


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        return a.ctypes.data, False
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), bool(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


def _as_host(a, dtype):
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def escape_status_str(code: int) -> str:
    return LIB.escape_status_str(int(code)).decode()


def escape_load_csr(n: int, row_ptr, col, flags: int = 0, stream=None):
    """Load a CSR (numpy host arrays or torch CUDA tensors); returns an opaque handle."""
    row_ptr = _as_host(row_ptr, np.int64)
    col = _as_host(col, np.int32)
    if isinstance(col, np.ndarray) and col.size == 0:
        col = np.zeros(1, dtype=np.int32)
        nnz = 0
    else:
        nnz = int(row_ptr[-1]) if isinstance(row_ptr, np.ndarray) else int(col.numel())
    prp, dev1 = _ptr(row_ptr)
    pcol, dev2 = _ptr(col)
    if dev1 != dev2:
        raise ValueError("row_ptr and col must both be host or both be device arrays")
    if dev1:
        flags |= ESCAPE_DEVICE_PTRS
    h = ctypes.c_void_p()
    _check(LIB.escape_load_csr(int(n), nnz, prp, pcol, int(flags), _stream(stream), ctypes.byref(h)),
           "escape_load_csr")
    return h


def escape_graph_info(h):
    n, m = ctypes.c_int64(), ctypes.c_int64()
    _check(LIB.escape_graph_info(h, ctypes.byref(n), ctypes.byref(m)), "escape_graph_info")
    return n.value, m.value


def escape_set_options(h, keep_per_element: bool = False, cta_per_sm: int = 0, serial_phases=None):
    """serial_phases: True / False, or None for the size-based default."""
    sp = -1 if serial_phases is None else int(bool(serial_phases))
    _check(LIB.escape_set_options(h, int(bool(keep_per_element)), int(cta_per_sm), sp), "escape_set_options")


def escape_census4(h, stream=None) -> dict:
    """The 3- and 4-vertex census alone (keys c3, c4, n3, n4)."""
    out = Census4()
    _check(LIB.escape_census4(h, ctypes.byref(out), _stream(stream)), "escape_census4")
    return out.to_dict()


def escape_census5(h, stream=None) -> dict:
    out = Census()
    _check(LIB.escape_census5(h, ctypes.byref(out), _stream(stream)), "escape_census5")
    return out.to_dict()


def escape_census5_batch(vtx_offsets, row_ptr, col, flags: int = 0, stream=None) -> list:
    vtx_offsets = _as_host(vtx_offsets, np.int64)
    row_ptr = _as_host(row_ptr, np.int64)
    col = _as_host(col, np.int32)
    if isinstance(col, np.ndarray) and col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    G = (len(vtx_offsets) if isinstance(vtx_offsets, np.ndarray) else int(vtx_offsets.numel())) - 1
    pv, d0 = _ptr(vtx_offsets)
    pr, d1 = _ptr(row_ptr)
    pc, d2 = _ptr(col)
    if not (d0 == d1 == d2):
        raise ValueError("batch arrays must all be host or all be device arrays")
    if d0:
        flags |= ESCAPE_DEVICE_PTRS
    out = (Census * max(G, 1))()
    _check(LIB.escape_census5_batch(int(G), pv, pr, pc, int(flags), out, _stream(stream)), "escape_census5_batch")
    return [out[k].to_dict() for k in range(G)]


def escape_per_element(h, stream=None) -> dict:
    n, m = escape_graph_info(h)
    nnz = 2 * m
    arrs = {k: np.zeros(max(nnz, 1), dtype=np.uint64) for k in ("T_e", "C4_e", "K4_e")}
    arrs.update({k: np.zeros(max(n, 1), dtype=np.uint64) for k in ("t_i", "C4_i", "K4_i")})
    _check(LIB.escape_per_element(h, arrs["T_e"].ctypes.data, arrs["C4_e"].ctypes.data, arrs["K4_e"].ctypes.data,
                                  arrs["t_i"].ctypes.data, arrs["C4_i"].ctypes.data, arrs["K4_i"].ctypes.data,
                                  _stream(stream)), "escape_per_element")
    return {k: (v[:nnz] if k.endswith("_e") else v[:n]) for k, v in arrs.items()}


def escape_last_phase_ms(h) -> dict:
    buf = (ctypes.c_float * N_PHASES)()
    k = LIB.escape_last_phase_ms(h, buf, N_PHASES)
    return {PHASE_NAMES[i]: float(buf[i]) for i in range(min(k, N_PHASES))}


def escape_last_kernel_launches(h) -> int:
    return int(LIB.escape_last_kernel_launches(h))


class Part(ctypes.Structure):
    _fields_ = [("sums", U128 * ESCAPE_PART_SUMS)]


def escape_part_sum_count() -> int:
    return int(LIB.escape_part_sum_count())


def escape_census5_part(h, part: int, parts: int, stream=None) -> list:
    """This part's raw sums of a census split over `parts` (Python ints, the
    first escape_part_sum_count() entries)."""
    out = Part()
    _check(LIB.escape_census5_part(h, int(part), int(parts), ctypes.byref(out), _stream(stream)),
           "escape_census5_part")
    k = escape_part_sum_count()
    return [int(out.sums[i].lo) | (int(out.sums[i].hi) << 64) for i in range(k)]


def escape_part_counts(h, k4_e=None, c4_e=None, c4_v=None, put: bool = False, stream=None):
    """Read (or, with put, write) the part's per-element arrays: uint64/int64
    numpy arrays or torch CUDA tensors of nnz, nnz and n entries."""
    ptrs = [_ptr(a) for a in (k4_e, c4_e, c4_v)]
    devs = {d for p, d in ptrs if p is not None}
    if len(devs) > 1:
        raise ValueError("arrays must all be host or all be device arrays")
    flags = (ESCAPE_DEVICE_PTRS if devs == {True} else 0) | (ESCAPE_PART_PUT if put else 0)
    _check(LIB.escape_part_counts(h, ptrs[0][0], ptrs[1][0], ptrs[2][0], flags, _stream(stream)),
           "escape_part_counts")


def escape_census5_finish(h, total_sums, stream=None) -> dict:
    """The census from every part's sums added (modulo 2^128) and the handle's
    per-element arrays holding every part's counts added."""
    tot = Part()
    mask = (1 << 64) - 1
    for i, v in enumerate(total_sums):
        v %= 1 << 128
        tot.sums[i].lo = v & mask
        tot.sums[i].hi = v >> 64
    out = Census()
    _check(LIB.escape_census5_finish(h, ctypes.byref(tot), ctypes.byref(out), _stream(stream)),
           "escape_census5_finish")
    return out.to_dict()


def escape_last_basis_counts(h) -> dict:
    """W, D, DP, DBP of the last escape_census5 call on the handle (Python ints)."""
    out = (U128 * 4)()
    _check(LIB.escape_last_basis_counts(h, out), "escape_last_basis_counts")
    vals = [int(x.lo) | (int(x.hi) << 64) for x in out]
    return dict(zip(("W", "D", "DP", "DBP"), vals))


def escape_cycles4_noalloc(n: int, row_ptr, col, c4_v, c4_total, stream=None):
    """Per-vertex 4-cycle counts into caller-provided device tensors, with no
    allocation inside the library (n <= ESCAPE_NOALLOC_MAX_N)."""
    ptrs = [_ptr(a) for a in (row_ptr, col, c4_v, c4_total)]
    if not all(dev for _, dev in ptrs):
        raise ValueError("escape_cycles4_noalloc takes device tensors only")
    _check(LIB.escape_cycles4_noalloc(int(n), ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], _stream(stream)),
           "escape_cycles4_noalloc")


ESCAPE_NOALLOC_MAX_N = 32768


def escape_free(h):
    if h:
        LIB.escape_free(h)


# ------------------------------------------------------------------ convenience

def census(row_ptr, col, n: int | None = None, flags: int = 0, per_element: bool = False, stream=None,
           four_only: bool = False) -> dict:
    """Load, count and free in one call.  Returns the census dict (plus
    'per_element' when asked); with four_only, the 3- and 4-vertex counts
    alone (escape_census4)."""
    if n is None:
        n = (len(row_ptr) if isinstance(row_ptr, np.ndarray) else int(row_ptr.numel())) - 1
    h = escape_load_csr(n, row_ptr, col, flags, stream)
    try:
        if per_element:
            escape_set_options(h, keep_per_element=True)
        out = escape_census4(h, stream) if four_only else escape_census5(h, stream)
        if per_element:
            out["per_element"] = escape_per_element(h, stream)
        out["phase_ms"] = escape_last_phase_ms(h)
        return out
    finally:
        escape_free(h)
