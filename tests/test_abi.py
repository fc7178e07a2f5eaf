"""CPU tests of the C ABI: the library builds for sm_103a, loads, exports every
entry point include/nq.h declares, and its host-side prefix generation equals
the oracle's. No call here launches a kernel."""
import ctypes
import json
import os

import numpy as np
import pytest

import synth_inputs
from paper_2511_12009_gb300 import nq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def to_state(n, cols_list):
    """Somers state (cols, ld, rd) of row d after queens at (r, cols_list[r]), r < d,
    from the board geometry: a queen at (r, c) attacks row d at c + (d - r) along one
    diagonal and c - (d - r) along the other."""
    d = len(cols_list)
    cols = sum(1 << int(c) for c in cols_list)
    ld = sum(1 << (int(c) + d - r) for r, c in enumerate(cols_list) if int(c) + d - r < n)
    rd = sum(1 << (int(c) - d + r) for r, c in enumerate(cols_list) if int(c) - d + r >= 0)
    return cols, ld, rd


def test_library_exports_every_declared_symbol():
    lib = nq.lib()
    syms = nq.header_symbols()
    assert len(syms) >= 10
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_strerror_names_every_code():
    for code in range(0, -8, -1):
        assert nq.strerror(code) and "unknown" not in nq.strerror(code)
    assert "unknown" in nq.strerror(-99)


@pytest.mark.parametrize("n,d", [(1, 0), (1, 1), (2, 2), (3, 2), (4, 2), (5, 1), (5, 2), (8, 3),
                                 (9, 4), (11, 5), (12, 0), (13, 3), (14, 3), (16, 5), (17, 4)])
def test_enumeration_equals_oracle(orc, n, d):
    got = nq.enumerate_prefixes(n, d)
    cols, w = orc.prefixes(n, d)
    assert len(got) == len(cols)
    for rec, q, wt in zip(got, cols, w):
        c, l, r = to_state(n, q)
        assert (int(rec["cols"]), int(rec["ld"]), int(rec["rd"])) == (c, l, r)
        meta = int(rec["meta"])
        assert meta & 3 == wt and (meta >> 2) & 31 == n and (meta >> 7) & 31 == d
        assert meta >> 12 == 0


@pytest.mark.parametrize("n,d", [(18, 5), (18, 6), (21, 5), (22, 5), (22, 6)])
def test_prefix_counts_equal_oracle(orc, n, d):
    assert nq.prefix_count(n, d) == orc.prefix_count(n, d)


def test_prefix_count_paper_n27():
    v = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["n27_subproblems"]
    assert nq.prefix_count(v["n"], v["d"]) == v["value"]


@pytest.mark.parametrize("n,d", [(10, 2), (12, 5), (13, 6), (16, 4)])
def test_ranks_equal_oracle(orc, n, d):
    total = nq.prefix_count(n, d)
    ranks = synth_inputs.sample_indices(11, total, 64) + [0, total - 1]
    got = nq.prefixes_at_ranks(n, d, ranks)
    want = orc.prefixes_at_ranks(n, d, ranks)
    for rec, q in zip(got, want):
        assert (int(rec["cols"]), int(rec["ld"]), int(rec["rd"])) == to_state(n, q)


def test_rank_out_of_range():
    with pytest.raises(nq.NQError) as e:
        nq.prefixes_at_ranks(8, 3, [nq.prefix_count(8, 3)])
    assert e.value.code == nq.NQ_EINVAL


def test_descendants_refine_in_order():
    n, d = 11, 3
    parents = nq.enumerate_prefixes(n, d)
    children = nq.enumerate_prefixes(n, d + 2)
    joined = np.concatenate([nq.descendants(p, 2) for p in parents])
    assert np.array_equal(joined, children)


def test_descendants_of_root_cover_the_board():
    # all 3-row placements of a 9x9 board, no symmetry (weight 1), by brute force
    kids = nq.descendants(nq.enumerate_prefixes(9, 0)[0], 3)
    brute = sum(1 for a in range(9) for b in range(9) for c in range(9)
                if len({a, b, c}) == 3 and abs(a - b) != 1 and abs(b - c) != 1 and abs(a - c) != 2)
    assert len(kids) == brute and all(int(k["meta"]) & 3 == 1 for k in kids)


@pytest.mark.parametrize("args", [(0, 0), (32, 3), (8, 9), (8, -1)])
def test_enumerate_rejects_bad_sizes(args):
    num = ctypes.c_uint64(0)
    assert nq.lib().nq_enumerate_prefixes(args[0], args[1], None, 0, ctypes.byref(num)) == nq.NQ_EINVAL


def test_enumerate_cap_too_small():
    """A buffer smaller than the set: NQ_EINVAL, the set's size in *n_out, nothing written."""
    out = np.zeros(3, dtype=nq.PREFIX_DTYPE)
    num = ctypes.c_uint64(0)
    rc = nq.lib().nq_enumerate_prefixes(8, 3, out.ctypes.data, 3, ctypes.byref(num))
    assert rc == nq.NQ_EINVAL and num.value == nq.prefix_count(8, 3)
    assert not out.view(np.uint32).any()
    parent = nq.enumerate_prefixes(9, 2)[0]
    kids = nq.descendants(parent, 2)
    par = np.ascontiguousarray(np.asarray(parent, dtype=nq.PREFIX_DTYPE).reshape(1))
    small = np.zeros(len(kids) - 1, dtype=nq.PREFIX_DTYPE)
    rc = nq.lib().nq_descendants(par.ctypes.data, 2, small.ctypes.data, len(small),
                                 ctypes.byref(num))
    assert rc == nq.NQ_EINVAL and num.value == len(kids) and not small.view(np.uint32).any()


@pytest.mark.parametrize("n", [20, 21, 22])
def test_sampled_ranks_equal_oracle_golden(n):
    """The library's unranking at the benchmark depth equals the oracle's prefixes
    stored with the seeded N=20..22 samples (tests/golden/make_golden.py)."""
    g = np.load(os.path.join(GOLDEN, f"oracle_n{n}_d7_s2048.npz"))
    got = nq.prefixes_at_ranks(n, 7, g["ranks"])
    assert np.array_equal(got["meta"] & 3, g["weights"])
    for rec, q in zip(got, g["cols"]):
        assert (int(rec["cols"]), int(rec["ld"]), int(rec["rd"])) == to_state(n, q)


def test_total_rejects_overflowing_sizes():
    out = ctypes.c_uint64(0)
    assert nq.lib().nq_total(29, ctypes.byref(out)) == nq.NQ_EOVERFLOW
    assert nq.lib().nq_total(0, ctypes.byref(out)) == nq.NQ_EINVAL


def test_default_depth_in_range():
    for n in range(1, 32):
        d = nq.default_depth(n)
        assert 0 <= d <= max(n - 2, 0)


def test_count_split_argument_errors():
    """Rejected on the host before any device work."""
    pre = nq.enumerate_prefixes(10, 3).copy()
    cnt = np.zeros(len(pre), dtype=np.uint64)
    lib = nq.lib()
    assert lib.nq_count_split(pre.ctypes.data, len(pre), 2, None, None, None, None, None,
                              None) == nq.NQ_EINVAL                       # no counts
    assert lib.nq_count_split(pre.ctypes.data, len(pre), -2, None, cnt.ctypes.data, None, None,
                              None, None) == nq.NQ_EINVAL                 # rows < -1
    assert lib.nq_count_split(pre.ctypes.data, (1 << 20) + 1, 2, None, cnt.ctypes.data, None,
                              None, None, None) == nq.NQ_EINVAL           # over the tag width
    bad = pre.copy()
    bad["cols"][0] |= np.uint32(1 << 12)                                  # off the board
    assert lib.nq_count_split(bad.ctypes.data, len(bad), 2, None, cnt.ctypes.data, None, None,
                              None, None) == nq.NQ_EINVAL
    tot = np.full(32, 7, dtype=np.uint64)
    assert lib.nq_count_split(None, 0, 2, None, cnt.ctypes.data, None, tot.ctypes.data, None,
                              None) == nq.NQ_OK
    assert int(tot.sum()) == 0
