"""CPU oracle for exact N-Queens counting -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package. The product package never imports
it, and it never imports the product package.

The arithmetic lives in ``nq_oracle.c`` (plain C, bool-array backtracker, no
bitmasks); this module only compiles it with gcc and marshals arguments through
ctypes. See the C file's header for what each function follows in the paper
(problem statement and symmetric decomposition of Section 1, the prefix
generation of Section 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ECAP = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile nq_oracle.c into oracle/_build/liboracle.so (gcc -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-pthread", "-Wall", "-Wextra", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i8p = ctypes.POINTER(ctypes.c_int8)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_brute_perm.argtypes = [ctypes.c_int, ip, u64p]
            lib.orc_total.argtypes = [ctypes.c_int, u64p, u64p]
            lib.orc_count_constrained.argtypes = [ctypes.c_int, ip, ip, ctypes.c_int, u64p, u64p]
            lib.orc_prefixes.argtypes = [ctypes.c_int, ctypes.c_int, i8p, u8p, ctypes.c_uint64, u64p]
            lib.orc_prefix_count.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
            lib.orc_prefixes_at_ranks.argtypes = [ctypes.c_int, ctypes.c_int, u64p,
                                                  ctypes.c_uint64, i8p, ctypes.c_int]
            lib.orc_count_prefixes.argtypes = [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_uint64,
                                               u64p, u64p, ctypes.c_int]
            for f in (lib.orc_brute_perm, lib.orc_total, lib.orc_count_constrained,
                      lib.orc_prefixes, lib.orc_prefix_count, lib.orc_prefixes_at_ranks,
                      lib.orc_count_prefixes):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _u128(pair) -> int:
    return int(pair[0]) | (int(pair[1]) << 64)


def _check(rc: int, what: str):
    if rc != ORC_OK:
        raise ValueError(f"oracle {what} failed with code {rc}")


def default_threads() -> int:
    return os.cpu_count() or 1


def brute_perm(n: int, fixed=None) -> int:
    """Count permutations with no two entries on a diagonal, by trying all N!.

    ``fixed`` is an optional list of length n with the forced column of each row
    or -1. N <= 12.
    """
    lib = _load()
    out = (ctypes.c_uint64 * 1)()
    fx = None
    if fixed is not None:
        fx = (ctypes.c_int * n)(*[int(v) for v in fixed])
    _check(lib.orc_brute_perm(n, fx, out), "brute_perm")
    return int(out[0])


def total(n: int) -> tuple[int, int]:
    """Q(N) and the node count of the full search, no symmetry. Returns (count, nodes)."""
    lib = _load()
    c = (ctypes.c_uint64 * 2)()
    v = (ctypes.c_uint64 * 2)()
    _check(lib.orc_total(n, c, v), "total")
    return _u128(c), _u128(v)


def count_constrained(n: int, queens) -> tuple[int, int]:
    """Solutions containing every (row, col) in ``queens``. Returns (count, nodes)."""
    lib = _load()
    k = len(queens)
    rows = (ctypes.c_int * max(k, 1))(*[int(q[0]) for q in queens])
    cols = (ctypes.c_int * max(k, 1))(*[int(q[1]) for q in queens])
    c = (ctypes.c_uint64 * 2)()
    v = (ctypes.c_uint64 * 2)()
    _check(lib.orc_count_constrained(n, rows, cols, k, c, v), "count_constrained")
    return _u128(c), _u128(v)


def prefix_count(n: int, d: int) -> int:
    """Size of the symmetric depth-d prefix set, counted without materialising it."""
    lib = _load()
    out = (ctypes.c_uint64 * 1)()
    _check(lib.orc_prefix_count(n, d, out), "prefix_count")
    return int(out[0])


def prefixes(n: int, d: int) -> tuple[np.ndarray, np.ndarray]:
    """The symmetric depth-d prefix set in canonical order.

    Returns (cols [num, d] int8 -- the column of the queen in each row 0..d-1,
    weights [num] uint8).
    """
    lib = _load()
    num = prefix_count(n, d)
    cols = np.zeros((max(num, 1), max(d, 1)), dtype=np.int8)
    w = np.zeros(max(num, 1), dtype=np.uint8)
    got = (ctypes.c_uint64 * 1)()
    _check(lib.orc_prefixes(n, d, _p(cols, ctypes.c_int8), _p(w, ctypes.c_uint8),
                            num, got), "prefixes")
    assert int(got[0]) == num
    return cols[:num, :d].copy(), w[:num].copy()


def prefixes_at_ranks(n: int, d: int, ranks, threads: int | None = None) -> np.ndarray:
    """Prefixes (column lists, [k, d] int8) at the given canonical indices."""
    lib = _load()
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.uint64))
    out = np.zeros((max(len(r), 1), max(d, 1)), dtype=np.int8)
    _check(lib.orc_prefixes_at_ranks(n, d, _p(r, ctypes.c_uint64), len(r),
                                     _p(out, ctypes.c_int8), threads or default_threads()),
           "prefixes_at_ranks")
    return out[:len(r), :d].copy()


def count_prefixes(n: int, cols: np.ndarray, threads: int | None = None
                   ) -> tuple[np.ndarray, np.ndarray]:
    """Per-prefix (solutions, nodes) as uint64 arrays, one entry per row of ``cols``."""
    lib = _load()
    cols = np.ascontiguousarray(cols, dtype=np.int8)
    num = cols.shape[0]
    d = cols.shape[1] if cols.ndim == 2 else 0
    counts = np.zeros(max(num, 1), dtype=np.uint64)
    nodes = np.zeros(max(num, 1), dtype=np.uint64)
    buf = cols if num else np.zeros((1, max(d, 1)), dtype=np.int8)
    _check(lib.orc_count_prefixes(n, d, _p(buf, ctypes.c_int8), num,
                                  _p(counts, ctypes.c_uint64), _p(nodes, ctypes.c_uint64),
                                  threads or default_threads()), "count_prefixes")
    return counts[:num].copy(), nodes[:num].copy()


def total_sym(n: int, d: int, threads: int | None = None) -> tuple[int, int]:
    """Q(N) through the symmetric decomposition: sum of weight x per-prefix count.

    Returns (count, nodes), nodes = the placements below the prefixes (rows d..N-1),
    unweighted -- the work the search does.
    """
    cols, w = prefixes(n, d)
    counts, nodes = count_prefixes(n, cols, threads)
    return (int(sum(int(a) * int(b) for a, b in zip(w, counts))),
            int(sum(int(x) for x in nodes)))


def descendants(n: int, cols_list, rows: int) -> list[tuple[int, ...]]:
    """All placements extending the queens cols_list (row r in column cols_list[r])
    by `rows` more rows, in canonical order (rows top-down, columns increasing),
    as column tuples. Plain Python: no symmetry rule applies below row 1."""
    base = [int(c) for c in cols_list]
    d = len(base)
    out: list[tuple[int, ...]] = []

    def free(placed, r, c):
        for rr, cc in enumerate(placed):
            if cc == c or abs(cc - c) == r - rr:
                return False
        return True

    def rec(placed):
        if len(placed) == d + rows:
            out.append(tuple(placed))
            return
        r = len(placed)
        for c in range(n):
            if free(placed, r, c):
                rec(placed + [c])

    rec(base)
    return out
