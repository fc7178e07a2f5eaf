"""Thin ctypes binding of libnq (include/nq.h): argument marshalling only.

Every step of the counting path runs inside libnq's CUDA kernels and host C++;
this module converts Python/numpy/torch arguments to pointers and sizes and
turns negative status codes into ``NQError``. PyTorch appears only as a holder
of device memory and streams. There is no fallback: if libnq.so cannot be
built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

NQ_OK, NQ_EINVAL, NQ_ENOMEM, NQ_ECUDA, NQ_EOVERFLOW, NQ_ETIMEOUT, NQ_ESTACK, NQ_EBUSY = (
    0, -1, -2, -3, -4, -5, -6, -7)
NQ_LAYOUT_DEFAULT, NQ_LAYOUT_PAPER, NQ_LAYOUT_REG, NQ_LAYOUT_WT = 0, 1, 2, 3
NQ_LAYOUT_WT32, NQ_LAYOUT_WT32A, NQ_LAYOUT_WTM, NQ_LAYOUT_REGM = 4, 5, 6, 7
NQ_LAYOUT_REGP, NQ_LAYOUT_REGZ, NQ_LAYOUT_REGPZ, NQ_LAYOUT_AVAIL = 8, 9, 10, 11
LAYOUTS = {"default": 0, "paper": 1, "reg": 2, "wt": 3, "wt32": 4, "wt32a": 5, "wtm": 6,
           "regm": 7, "regp": 8, "regz": 9, "regpz": 10, "avail": 11}
NQ_MAX_N = 31

# numpy view of nq_prefix {u32 cols, ld, rd, meta}
PREFIX_DTYPE = np.dtype([("cols", "<u4"), ("ld", "<u4"), ("rd", "<u4"), ("meta", "<u4")])


class NQError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class Config(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int32), ("block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("order", ctypes.c_int32),
                ("d", ctypes.c_int32), ("claim", ctypes.c_int32),
                ("donate", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Timing(ctypes.Structure):
    _fields_ = [("enumerate_ms", ctypes.c_double), ("upload_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("prefixes", ctypes.c_uint64), ("d", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("block", ctypes.c_int32), ("grid", ctypes.c_int32)]


class Queen(ctypes.Structure):
    _fields_ = [("row", ctypes.c_int8), ("col", ctypes.c_int8)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int


def _declare(lib):
    sig = {
        "nq_enumerate_prefixes": (_i32, [_i32, _i32, _vp, _u64, ctypes.POINTER(_u64)]),
        "nq_prefixes_at_ranks": (_i32, [_i32, _i32, _vp, _u64, _vp]),
        "nq_descendants": (_i32, [_vp, _i32, _vp, _u64, ctypes.POINTER(_u64)]),
        "nq_default_depth": (_i32, [_i32]),
        "nq_count": (_i32, [_i32, _i32, _vp, _u64, _vp, _vp]),
        "nq_count_ex": (_i32, [_vp, _u64, _i32, _i32, _vp, _vp, _vp, ctypes.POINTER(Config), _vp]),
        "nq_sync": (_i32, [_vp]),
        "nq_total": (_i32, [_i32, ctypes.POINTER(_u64)]),
        "nq_total_ex": (_i32, [_i32, ctypes.POINTER(Config), ctypes.POINTER(_u64),
                               ctypes.POINTER(_u64), ctypes.POINTER(Timing)]),
        "nq_count_split": (_i32, [_vp, _u64, _i32, ctypes.POINTER(Config), _vp, _vp, _vp,
                                  ctypes.POINTER(_i32), ctypes.POINTER(Timing)]),
        "nq_count_constrained": (_i32, [_i32, ctypes.POINTER(Queen), _i32, ctypes.POINTER(_u64)]),
        "nq_strerror": (ctypes.c_char_p, [_i32]),
        "nq_probe_alu": (_i32, [_i32, _i32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "nq_batch_create": (_i32, [ctypes.POINTER(_i32), ctypes.POINTER(_i32), _i32,
                                   ctypes.POINTER(Config), ctypes.POINTER(_vp)]),
        "nq_batch_info": (_i32, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_i32),
                                 ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
        "nq_batch_run": (_i32, [_vp, _vp, ctypes.POINTER(_u64), ctypes.POINTER(ctypes.c_float)]),
        "nq_batch_run_separate": (_i32, [_vp, _vp, ctypes.POINTER(_u64),
                                         ctypes.POINTER(ctypes.c_float)]),
        "nq_batch_counts": (_i32, [_vp, _i32, _vp, _u64, ctypes.POINTER(_u64)]),
        "nq_batch_destroy": (None, [_vp]),
        "nq_probe_smem": (_i32, [_i32, ctypes.c_uint32, _i32, _i32, _i32,
                                 ctypes.POINTER(ctypes.c_double)]),
        "nq_stack_offset": (_i32, [_i32, _i32, _i32, _i32, _i32, _i32,
                                   ctypes.POINTER(ctypes.c_uint32)]),
        "nq_partition": (_i32, [_u64, _vp, _i32, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib():
    """Load libnq.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            handle = ctypes.CDLL(path)
            _declare(handle)
            _lib = handle
    return _lib


def library_path() -> str:
    return _build.LIB


def strerror(code: int) -> str:
    return lib().nq_strerror(int(code)).decode()


def _check(rc: int, what: str):
    if rc != NQ_OK:
        raise NQError(rc, what)


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_config(layout=0, block=0, blocks_per_sm=0, order=0, d=0, claim=0, donate=0) -> Config:
    if isinstance(layout, str):
        layout = LAYOUTS[layout]
    return Config(int(layout), int(block), int(blocks_per_sm), int(order), int(d), int(claim),
                  int(donate), 0)


# --- host prefix generation --------------------------------------------------

def default_depth(n: int) -> int:
    d = lib().nq_default_depth(int(n))
    if d < 0:
        raise NQError(d, "nq_default_depth")
    return d


def prefix_count(n: int, d: int) -> int:
    num = _u64(0)
    _check(lib().nq_enumerate_prefixes(int(n), int(d), None, 0, ctypes.byref(num)),
           "nq_enumerate_prefixes")
    return int(num.value)


def enumerate_prefixes(n: int, d: int) -> np.ndarray:
    """Symmetric depth-d prefix set, canonical order, as a PREFIX_DTYPE array."""
    num = prefix_count(n, d)
    out = np.zeros(max(num, 1), dtype=PREFIX_DTYPE)
    got = _u64(0)
    _check(lib().nq_enumerate_prefixes(int(n), int(d), out.ctypes.data, num, ctypes.byref(got)),
           "nq_enumerate_prefixes")
    return out[:num]


def prefixes_at_ranks(n: int, d: int, ranks) -> np.ndarray:
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.uint64))
    out = np.zeros(max(len(r), 1), dtype=PREFIX_DTYPE)
    _check(lib().nq_prefixes_at_ranks(int(n), int(d), r.ctypes.data, len(r), out.ctypes.data),
           "nq_prefixes_at_ranks")
    return out[:len(r)]


def descendants(parent: np.ndarray, rows: int) -> np.ndarray:
    par = np.ascontiguousarray(np.asarray(parent, dtype=PREFIX_DTYPE).reshape(1))
    num = _u64(0)
    _check(lib().nq_descendants(par.ctypes.data, int(rows), None, 0, ctypes.byref(num)),
           "nq_descendants")
    out = np.zeros(max(num.value, 1), dtype=PREFIX_DTYPE)
    got = _u64(0)
    _check(lib().nq_descendants(par.ctypes.data, int(rows), out.ctypes.data, num.value,
                                ctypes.byref(got)), "nq_descendants")
    return out[:num.value]


# --- device search -------------------------------------------------------------

def to_device(prefixes: np.ndarray, device="cuda"):
    """Copy a PREFIX_DTYPE array into a torch int32 [n, 4] device tensor."""
    import torch
    arr = np.ascontiguousarray(prefixes, dtype=PREFIX_DTYPE).view(np.int32).reshape(-1, 4)
    return torch.from_numpy(arr.copy()).to(device)


def _ptr(t):
    return None if t is None else t.data_ptr()


def count(n: int, d: int, d_prefixes, d_counts, stream=None):
    """Enqueue nq_count: d_prefixes int32 [m, 4] device tensor, d_counts int64 [m] device tensor."""
    m = int(d_prefixes.shape[0])
    _check(lib().nq_count(int(n), int(d), _ptr(d_prefixes), m, _ptr(d_counts),
                          _stream_handle(stream)), "nq_count")


def count_ex(d_prefixes, min_d: int, max_n: int, d_counts=None, d_nodes=None, d_totals=None,
             config: Config | None = None, stream=None):
    m = int(d_prefixes.shape[0])
    cfg = ctypes.byref(config) if config is not None else None
    _check(lib().nq_count_ex(_ptr(d_prefixes), m, int(min_d), int(max_n), _ptr(d_counts),
                             _ptr(d_nodes), _ptr(d_totals), cfg, _stream_handle(stream)),
           "nq_count_ex")


def sync(stream=None):
    _check(lib().nq_sync(_stream_handle(stream)), "nq_sync")


def total(n: int) -> int:
    out = _u64(0)
    _check(lib().nq_total(int(n), ctypes.byref(out)), "nq_total")
    return int(out.value)


def total_ex(n: int, config: Config | None = None, nodes: bool = False) -> dict:
    out = _u64(0)
    nod = _u64(0)
    tm = Timing()
    cfg = ctypes.byref(config) if config is not None else None
    _check(lib().nq_total_ex(int(n), cfg, ctypes.byref(out), ctypes.byref(nod) if nodes else None,
                             ctypes.byref(tm)), "nq_total_ex")
    res = {"total": int(out.value), "enumerate_ms": tm.enumerate_ms, "upload_ms": tm.upload_ms,
           "kernel_ms": tm.kernel_ms, "total_ms": tm.total_ms, "prefixes": int(tm.prefixes),
           "d": tm.d, "layout": tm.layout, "block": tm.block, "grid": tm.grid}
    if nodes:
        res["nodes"] = int(nod.value)
    return res


def count_split(prefixes: np.ndarray, rows: int = -1, config: Config | None = None,
                nodes: bool = False) -> dict:
    """nq_count_split on host records: per-prefix counts (and nodes), per-N
    weighted totals, the rows added and the call's timing."""
    pre = np.ascontiguousarray(prefixes, dtype=PREFIX_DTYPE)
    n = len(pre)
    counts = np.zeros(max(n, 1), dtype=np.uint64)
    nod = np.zeros(max(n, 1), dtype=np.uint64) if nodes else None
    totals = np.zeros(32, dtype=np.uint64)
    used = _i32(0)
    tm = Timing()
    cfg = ctypes.byref(config) if config is not None else None
    _check(lib().nq_count_split(pre.ctypes.data if n else None, n, int(rows), cfg,
                                counts.ctypes.data, nod.ctypes.data if nodes else None,
                                totals.ctypes.data, ctypes.byref(used), ctypes.byref(tm)),
           "nq_count_split")
    res = {"counts": counts[:n], "totals": totals, "rows": int(used.value),
           "children": int(tm.prefixes), "split_ms": tm.enumerate_ms, "upload_ms": tm.upload_ms,
           "kernel_ms": tm.kernel_ms, "total_ms": tm.total_ms, "layout": tm.layout,
           "block": tm.block, "grid": tm.grid}
    if nodes:
        res["nodes"] = nod[:n]
    return res


def count_constrained(n: int, queens) -> int:
    k = len(queens)
    arr = (Queen * max(k, 1))(*[Queen(int(r), int(c)) for r, c in queens])
    out = _u64(0)
    _check(lib().nq_count_constrained(int(n), arr, k, ctypes.byref(out)), "nq_count_constrained")
    return int(out.value)


def probe_alu(kind: int, iters: int = 4096) -> dict:
    """Integer issue-rate microbenchmark (see nq_probe_alu in include/nq.h)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().nq_probe_alu(int(kind), int(iters), ctypes.byref(a), ctypes.byref(b),
                              ctypes.byref(c)), "nq_probe_alu")
    return {"per_clk_per_sm": a.value, "per_s": b.value, "sm_mhz": c.value}


def probe_smem(kind: int, lane_mask: int = 0xFFFFFFFF, density: int = 32, iters: int = 256,
               slots: int = 8) -> float:
    """Shared-memory pattern probe (nq_probe_smem); returns the launch time in ms."""
    ms = ctypes.c_double()
    _check(lib().nq_probe_smem(int(kind), int(lane_mask) & 0xFFFFFFFF, int(density), int(iters),
                               int(slots), ctypes.byref(ms)), "nq_probe_smem")
    return ms.value


def stack_offset(layout, block: int, slots: int, thread: int, slot: int, field: int) -> int:
    """Byte offset of a stack word in the search kernel's shared memory (nq_stack_offset)."""
    if isinstance(layout, str):
        layout = LAYOUTS[layout]
    out = ctypes.c_uint32()
    _check(lib().nq_stack_offset(int(layout), int(block), int(slots), int(thread), int(slot),
                                 int(field), ctypes.byref(out)), "nq_stack_offset")
    return int(out.value)


def partition(n: int, k: int, ratios=None) -> list[tuple[int, int]]:
    """Static split of n subproblems over k workers (nq_partition): [(first, count)]."""
    first = np.zeros(max(k, 1), dtype=np.uint64)
    count = np.zeros(max(k, 1), dtype=np.uint64)
    rp = None
    if ratios is not None:
        r = np.ascontiguousarray(np.asarray(ratios, dtype=np.float32))
        if len(r) != k:
            raise ValueError("one ratio per worker")
        rp = r.ctypes.data
    _check(lib().nq_partition(int(n), rp, int(k), first.ctypes.data, count.ctypes.data),
           "nq_partition")
    return [(int(f), int(c)) for f, c in zip(first, count)]


def header_symbols() -> list[str]:
    """Entry points declared in include/nq.h (for the export check)."""
    import re
    path = os.path.join(_build.INCLUDE, "nq.h")
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(nq_\w+)\s*\(", text, re.M)))
