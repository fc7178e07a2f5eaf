"""Pins for the CPU oracle, against things other than the oracle itself.

Every pin here is one of: brute force over all permutations or all partial
placements (tiny N), a published table of the plain definition (OEIS A000170),
a value the paper prints (Section 4.5 log), a board-symmetry invariant, or a
structural identity of the prefix decomposition (Section 1). A plausible
mistake in the oracle -- a missed diagonal, a wrong row-0 half, a wrong
odd-N centre rule, an off-by-one in the node count or in the prefix order --
fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import synth_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _json(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --- independent brute force written in Python from the definition -------

def _nonattacking(cols):
    """cols[r] = column of the queen in row r; True if no two share a column/diagonal."""
    for i in range(len(cols)):
        for j in range(i + 1, len(cols)):
            if cols[i] == cols[j] or abs(cols[i] - cols[j]) == j - i:
                return False
    return True


def _py_count(n, fixed=None):
    """Solutions by enumerating all n! permutations."""
    total = 0
    for perm in itertools.permutations(range(n)):
        if fixed and any(perm[r] != c for r, c in fixed.items()):
            continue
        if _nonattacking(perm):
            total += 1
    return total


def _py_partial(n, k):
    """Number of non-attacking placements of queens in rows 0..k-1 (brute force over n^k)."""
    return sum(1 for t in itertools.product(range(n), repeat=k) if _nonattacking(t))


# --- totals ----------------------------------------------------------------

@pytest.mark.parametrize("n", range(0, 11))
def test_brute_force_c_equals_backtracker(orc, n):
    assert orc.brute_perm(n) == orc.total(n)[0]


@pytest.mark.parametrize("n", range(1, 8))
def test_python_brute_force_equals_backtracker(orc, n):
    assert _py_count(n) == orc.total(n)[0]


def test_oeis_table_small(orc):
    q = _json("oeis_a000170.json")["Q"]
    for n in range(1, 14):
        assert orc.total(n)[0] == q[str(n)], n


def test_oeis_table_symmetric_driver(orc):
    q = _json("oeis_a000170.json")["Q"]
    for n, d in [(14, 3), (15, 4), (16, 5)]:
        assert orc.total_sym(n, d)[0] == q[str(n)], n


def test_paper_q27_fits_u64_and_matches_record():
    paper = _json("paper_values.json")["q27"]["value"]
    q = _json("oeis_a000170.json")["Q"]
    assert paper == q["27"]
    assert paper < 2 ** 63
    # the paper's own projection (Section 4.5) uses Q27/Q26 ~ 10.52
    assert abs(paper / q["26"] - 10.52) < 0.01


# --- node count definition ------------------------------------------------

@pytest.mark.parametrize("n", range(1, 8))
def test_nodes_equal_partial_placements(orc, n):
    # a node is one successful placement in some row; the full search from the
    # empty board visits every non-attacking placement of rows 0..k-1 once
    expect = sum(_py_partial(n, k) for k in range(1, n + 1))
    assert orc.total(n)[1] == expect


# --- symmetric decomposition (Section 1) -----------------------------------

@pytest.mark.parametrize("n", range(1, 13))
def test_symmetric_equals_plain(orc, n):
    q = orc.total(n)[0]
    for d in range(0, min(n, 6) + 1):
        assert orc.total_sym(n, d)[0] == q, (n, d)


def test_prefix_counts_survey_and_paper(orc):
    paper = _json("paper_values.json")["n27_subproblems"]
    assert orc.prefix_count(paper["n"], paper["d"]) == paper["value"]


@pytest.mark.parametrize("n,d", [(5, 2), (8, 3), (9, 3), (11, 4), (12, 2), (13, 1), (7, 7)])
def test_prefix_set_by_brute_force(orc, n, d):
    """The prefix set equals the brute-force set of non-attacking d-row placements
    with row 0 in the left half (or the centre column for odd N, the row-1 queen
    then in columns 0..m-2 when d >= 2), in lexicographic order."""
    m = n // 2
    want, wts = [], []
    for t in itertools.product(range(n), repeat=d):
        if not _nonattacking(t):
            continue
        if d == 0:
            want.append(t), wts.append(1)
            continue
        if t[0] < m:
            want.append(t), wts.append(2)
        elif n % 2 == 1 and t[0] == m:
            if d == 1:
                want.append(t), wts.append(1)
            elif t[1] <= m - 2:
                want.append(t), wts.append(2)
    # lexicographic order with the centre branch last is canonical order
    cols, w = orc.prefixes(n, d)
    assert [tuple(int(x) for x in row) for row in cols] == want
    assert list(w) == wts


@pytest.mark.parametrize("n", [6, 7, 10, 11])
def test_refinement_identity(orc, n):
    """For d >= 2, the (d+1)-prefixes are the children of the d-prefixes in order,
    and each prefix's count and nodes are the sums over its children."""
    for d in (2, 3):
        cp, wp = orc.prefixes(n, d)
        cc, wc = orc.prefixes(n, d + 1)
        kp, vp = orc.count_prefixes(n, cp)
        kc, vc = orc.count_prefixes(n, cc)
        j = 0
        for i in range(len(cp)):
            s_count, s_nodes = 0, 0
            while j < len(cc) and tuple(cc[j][:d]) == tuple(cp[i]):
                assert wc[j] == wp[i]
                s_count += int(kc[j])
                s_nodes += 1 + int(vc[j])
                j += 1
            assert s_count == int(kp[i])
            assert s_nodes == int(vp[i])
        assert j == len(cc)


def test_mirror_invariance(orc):
    n, d = 11, 4
    cols, _ = orc.prefixes(n, d)
    a, na = orc.count_prefixes(n, cols)
    b, nb = orc.count_prefixes(n, (n - 1 - cols.astype(np.int16)).astype(np.int8))
    assert np.array_equal(a, b) and np.array_equal(na, nb)


def test_invalid_prefix_rejected(orc):
    with pytest.raises(ValueError):
        orc.count_prefixes(6, np.array([[0, 1]], dtype=np.int8))  # diagonal neighbours


def test_degenerate_sizes(orc):
    assert orc.prefixes(2, 2)[0].shape == (0, 2)          # no 2-row prefix on a 2x2 board
    assert orc.total_sym(1, 1) == (1, 0)                    # centre prefix, weight 1
    assert orc.total_sym(3, 2)[0] == 0
    c, _ = orc.prefixes(8, 8)                               # d = N: the prefixes are solutions
    assert len(c) == 46 and orc.count_prefixes(8, c)[0].tolist() == [1] * 46


# --- unranking ---------------------------------------------------------------

@pytest.mark.parametrize("n,d", [(6, 2), (9, 3), (10, 5), (11, 6), (12, 7), (13, 4)])
def test_unranking_matches_enumeration(orc, n, d):
    cols, _ = orc.prefixes(n, d)
    ranks = synth_inputs.sample_indices(7, len(cols), 40) + [0, len(cols) - 1]
    got = orc.prefixes_at_ranks(n, d, ranks)
    assert np.array_equal(got, cols[ranks])


def test_unranking_out_of_range(orc):
    with pytest.raises(ValueError):
        orc.prefixes_at_ranks(8, 3, [orc.prefix_count(8, 3)])


# --- constrained counts --------------------------------------------------------

def test_constrained_zero_queens_is_total(orc):
    for n in range(1, 10):
        assert orc.count_constrained(n, [])[0] == orc.total(n)[0]


@pytest.mark.parametrize("seed", range(6))
def test_constrained_vs_brute_force(orc, seed):
    g = synth_inputs.SplitMix64(100 + seed)
    for _ in range(8):
        n = 4 + g.below(5)                     # 4..8
        k = g.below(4)
        qs = synth_inputs.constraint_set(g, n, k)
        fixed = {r: c for r, c in qs}
        want = _py_count(n, fixed)
        got = orc.count_constrained(n, qs)[0]
        assert got == want, (n, qs)
        fx = [-1] * n
        for r, c in qs:
            fx[r] = c
        assert orc.brute_perm(n, fx) == want


def _dihedral(n):
    f = n - 1
    return [lambda r, c: (r, c), lambda r, c: (c, f - r), lambda r, c: (f - r, f - c),
            lambda r, c: (f - c, r), lambda r, c: (r, f - c), lambda r, c: (f - r, c),
            lambda r, c: (c, r), lambda r, c: (f - c, f - r)]


@pytest.mark.parametrize("seed", range(3))
def test_constrained_board_symmetry(orc, seed):
    g = synth_inputs.SplitMix64(200 + seed)
    n = 9 + g.below(2)
    qs = synth_inputs.constraint_set(g, n, 1 + g.below(3))
    base = orc.count_constrained(n, qs)[0]
    for t in _dihedral(n):
        assert orc.count_constrained(n, [t(r, c) for r, c in qs])[0] == base


def test_constrained_conflicts_and_errors(orc):
    assert orc.count_constrained(8, [(0, 0), (1, 1)])[0] == 0   # diagonal attack
    assert orc.count_constrained(8, [(0, 0), (0, 3)])[0] == 0   # two in one row
    assert orc.count_constrained(8, [(0, 0), (5, 0)])[0] == 0   # same column
    one = orc.count_constrained(8, [(2, 5)])[0]
    assert orc.count_constrained(8, [(2, 5), (2, 5)])[0] == one  # duplicate cell
    with pytest.raises(ValueError):
        orc.count_constrained(8, [(8, 0)])
    with pytest.raises(ValueError):
        orc.count_constrained(8, [(0, -1)])


@pytest.mark.parametrize("n,base,rows", [(6, [], 3), (7, [1], 2), (8, [0, 2], 3), (9, [4, 0, 7], 2)])
def test_descendants_by_brute_force(orc, n, base, rows):
    """Extensions of a placement by `rows` rows: brute force over all column tuples."""
    want = [tuple(base) + t for t in itertools.product(range(n), repeat=rows)
            if _nonattacking(tuple(base) + t)]
    assert orc.descendants(n, base, rows) == want


@pytest.mark.parametrize("n,fname", [(20, "oracle_n20_d7_s2048.npz"), (21, "oracle_n21_d7_s2048.npz"),
                                     (22, "oracle_n22_d7_s2048.npz")])
def test_sampled_goldens_follow_their_recipe(orc, n, fname):
    """The stored N=20..22 samples are what their recipe says: the seeded ranks
    (SplitMix64 draws over the oracle's set size), the oracle's own prefixes at
    those ranks, every weight 2 (d >= 2), and -- re-derived here for the first
    entries, whole-board brute force being out of reach -- the oracle's counts;
    every count is at most the entry's node count (each solution is a node)."""
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", fname))
    size = orc.prefix_count(n, 7)
    assert int(g["set_size"][0]) == size
    ranks = synth_inputs.sample_ranks(int(g["seed"][0]), size, len(g["ranks"]))
    assert np.array_equal(g["ranks"], np.array(ranks, dtype=np.uint64))
    head = orc.prefixes_at_ranks(n, 7, g["ranks"][:64])
    assert np.array_equal(g["cols"][:64], head)
    assert (g["weights"] == 2).all()
    k = 4 if n < 22 else 2
    c, v = orc.count_prefixes(n, g["cols"][:k])
    assert np.array_equal(c, g["counts"][:k]) and np.array_equal(v, g["nodes"][:k])
    assert (g["counts"] <= g["nodes"]).all()
