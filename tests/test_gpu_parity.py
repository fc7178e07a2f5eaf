"""GPU parity: libnq's CUDA search against the CPU oracle, element by element.

Counts are integers, so the bar is bit-exact equality for every per-prefix
count, every per-prefix node count and every total. Inputs are the canonical
prefix sets (seeded samples where the oracle cannot cover a whole set), on
sizes that span many warps and blocks with ragged tails, plus the degenerate
cases (empty batch, prefixes that already are solutions, one row left, dead
prefixes, the whole board as one prefix).
"""
import json
import os

import numpy as np
import pytest

import synth_inputs
from paper_2511_12009_gb300 import nq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = {int(k): v for k, v in json.load(open(os.path.join(GOLDEN, "oeis_a000170.json")))["Q"].items()}
LAYOUTS = ["paper", "reg", "wt", "wt32", "wt32a", "wtm", "regm", "regp", "regz", "regpz",
           "avail"]
SPLIT_WORDS = {"regz", "regpz"}  # compiled for 256-thread blocks


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nq.lib()


_ORACLE = {}


def oracle_counts(orc, n, d):
    """Per-prefix (counts, nodes) of the canonical depth-d set, cached per (N, d)."""
    if (n, d) not in _ORACLE:
        _ORACLE[(n, d)] = orc.count_prefixes(n, orc.prefixes(n, d)[0])
    return _ORACLE[(n, d)]


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def run(pre, min_d, max_n, layout="reg", nodes=False, **cfg):
    dp = nq.to_device(pre)
    m = len(pre)
    cnt = torch.full((max(m, 1),), -1, dtype=torch.int64, device="cuda")
    nod = torch.full((max(m, 1),), -1, dtype=torch.int64, device="cuda") if nodes else None
    tot = torch.zeros(32, dtype=torch.int64, device="cuda")
    nq.count_ex(dp, min_d, max_n, cnt, nod, tot, nq.make_config(layout, **cfg))
    nq.sync()
    return u64(cnt)[:m], (u64(nod)[:m] if nodes else None), u64(tot)


def weighted(pre, counts):
    return int(sum(int(m & 3) * int(c) for m, c in zip(pre["meta"], counts)))


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("n,d", [(1, 0), (1, 1), (2, 1), (3, 1), (4, 2), (5, 1), (5, 2), (6, 0),
                                 (7, 3), (8, 0), (8, 3), (9, 2), (10, 4), (11, 3), (12, 4), (13, 5),
                                 (14, 3), (14, 6), (15, 5), (16, 5)])
def test_per_prefix_counts_and_nodes(orc, layout, n, d):
    pre = nq.enumerate_prefixes(n, d)
    want_c, want_n = oracle_counts(orc, n, d)
    got_c, got_n, tot = run(pre, d, n, layout, nodes=True)
    assert np.array_equal(got_c, want_c)
    assert np.array_equal(got_n, want_n)
    assert int(tot[n]) == Q[n] == weighted(pre, got_c)
    # the production build (no node counters) gives the same counts
    got_c2, _, tot2 = run(pre, d, n, layout)
    assert np.array_equal(got_c2, want_c) and int(tot2[n]) == Q[n]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("n", [16, 17, 18])
def test_full_board_golden(layout, n):
    """Every one of the d=5 prefixes' counts and nodes, against arrays the oracle wrote."""
    g = np.load(os.path.join(GOLDEN, f"oracle_n{n}_d5.npz"))
    pre = nq.enumerate_prefixes(n, 5)
    assert np.array_equal(pre["meta"] & 3, g["weights"])
    got_c, got_n, tot = run(pre, 5, n, layout, nodes=True)
    assert np.array_equal(got_c, g["counts"])
    assert np.array_equal(got_n, g["nodes"])
    assert int(tot[n]) == Q[n]
    got_c2, _, tot2 = run(pre, 5, n, layout)
    assert np.array_equal(got_c2, g["counts"]) and int(tot2[n]) == Q[n]


@pytest.mark.parametrize("n", list(range(1, 21)))
def test_total_public_entry(n):
    assert nq.total(n) == Q[n]


@pytest.mark.parametrize("n,d", [(16, 8), (17, 6), (18, 8), (12, 9), (13, 13), (19, 4), (11, 1)])
def test_total_ex_pieces(n, d):
    """nq_total_ex writes, uploads and searches large prefix sets in pieces
    (heaviest first, one stream each); small sets in one piece. Every depth,
    including the deepest (the whole board placed) and one row (odd N: the centre prefix
    alone has weight 1), gives Q(N)."""
    r = nq.total_ex(n, nq.make_config(d=d))
    assert r["total"] == Q[n] and r["prefixes"] == nq.prefix_count(n, d)


def test_environment_defaults(monkeypatch):
    """Unset configuration fields take NQ_LAYOUT / NQ_BLOCK / NQ_D from the
    environment; fields the caller sets win; bad values are ignored."""
    monkeypatch.setenv("NQ_LAYOUT", "reg")
    monkeypatch.setenv("NQ_BLOCK", "128")
    monkeypatch.setenv("NQ_D", "6")
    r = nq.total_ex(16)
    assert (r["total"], r["layout"], r["block"], r["d"]) == (Q[16], 2, 128, 6)
    r = nq.total_ex(16, nq.make_config("wt", 256, d=5))
    assert (r["total"], r["layout"], r["block"], r["d"]) == (Q[16], 3, 256, 5)
    monkeypatch.setenv("NQ_LAYOUT", "no-such-layout")
    monkeypatch.setenv("NQ_BLOCK", "-5")
    monkeypatch.delenv("NQ_D")
    r = nq.total_ex(16)
    # defaults: layout REGP, the block size that keeps the most threads resident
    assert (r["total"], r["layout"]) == (Q[16], nq.LAYOUTS["regp"])
    assert r["block"] in (128, 160, 192, 224, 256)
    assert r["d"] == nq.default_depth(16)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_launch_shapes(orc, layout):
    """Block sizes, blocks per SM and claim order do not change any count."""
    n, d = 13, 4
    pre = nq.enumerate_prefixes(n, d)
    want, _ = oracle_counts(orc, n, d)
    shapes = [(32, 1, 0), (64, 3, 1), (128, 0, 2), (512, 1, 1), (1024, 0, 0)]
    if layout in SPLIT_WORDS:
        shapes = [(256, 1, 0), (256, 3, 1), (256, 0, 2)]
    for block, bps, order in shapes:
        got, _, tot = run(pre, d, n, layout, block=block, blocks_per_sm=bps, order=order)
        assert np.array_equal(got, want), (block, bps, order)
        assert int(tot[n]) == Q[n]


def test_sampled_prefixes_at_bench_shape(orc):
    """N=18 at the library's default depth, in the default launch: 256 seeded
    prefixes, each checked one by one against the oracle."""
    n = 18
    d = nq.default_depth(n)
    pre = nq.enumerate_prefixes(n, d)
    got, _, tot = run(pre, d, n, "default")
    assert int(tot[n]) == Q[n]
    idx = synth_inputs.sample_indices(2024, len(pre), 256)
    cols, _ = orc.prefixes(n, d)
    want, _ = orc.count_prefixes(n, cols[idx])
    assert np.array_equal(got[idx], want)


def test_mixed_board_sizes_one_launch(orc):
    """Prefixes of N=6..14 interleaved in one launch: per-prefix counts and per-N totals."""
    parts, want = [], []
    for n in range(6, 15):
        d = 3
        parts.append(nq.enumerate_prefixes(n, d))
        want.append(orc.count_prefixes(n, orc.prefixes(n, d)[0])[0])
    pre = np.concatenate(parts)
    perm = np.random.default_rng(5).permutation(len(pre))
    got, _, tot = run(pre[perm], 3, 14)
    assert np.array_equal(got, np.concatenate(want)[perm])
    for n in range(6, 15):
        assert int(tot[n]) == Q[n]


def test_empty_batch():
    pre = nq.enumerate_prefixes(2, 2)
    assert len(pre) == 0
    got, _, tot = run(pre, 2, 2)
    assert len(got) == 0 and int(tot.sum()) == 0


@pytest.mark.parametrize("layout", LAYOUTS)
def test_degenerate_prefixes(orc, layout):
    """d = N (the prefixes are solutions), d = N - 1 (one row left), and
    prefixes whose next row is already dead."""
    for n in (6, 8, 9):
        for d in (n, n - 1, n - 2):
            pre = nq.enumerate_prefixes(n, d)
            want, want_n = oracle_counts(orc, n, d)
            got, got_n, tot = run(pre, d, n, layout, nodes=True)
            assert np.array_equal(got, want) and np.array_equal(got_n, want_n)
            assert int(tot[n]) == Q[n]


def random_placements(n, d, k, seed):
    """k seeded random non-attacking placements of rows 0..d-1 on an n x n board
    (each row a uniform choice among its free columns, restarting at a dead end)."""
    g = synth_inputs.SplitMix64(seed)
    out = []
    while len(out) < k:
        placed = []
        for r in range(d):
            free = [c for c in range(n)
                    if all(c != pc and abs(c - pc) != r - pr for pr, pc in enumerate(placed))]
            if not free:
                break
            placed.append(free[g.below(len(free))])
        if len(placed) == d:
            out.append(placed)
    return out


def records_of(n, placements):
    """Subproblem records (weight 1) from column lists, by the board geometry: a
    queen at (r, c) attacks row d at c + (d - r) and c - (d - r)."""
    pre = np.zeros(len(placements), dtype=nq.PREFIX_DTYPE)
    for i, q in enumerate(placements):
        d = len(q)
        pre[i]["cols"] = sum(1 << c for c in q)
        pre[i]["ld"] = sum(1 << (c + d - r) for r, c in enumerate(q) if c + d - r < n)
        pre[i]["rd"] = sum(1 << (c - d + r) for r, c in enumerate(q) if c - d + r >= 0)
        pre[i]["meta"] = 1 | (n << 2) | (d << 7)
    return pre


@pytest.mark.parametrize("layout", ["regm", "reg", "paper", "regp", "regz", "regpz"])
@pytest.mark.parametrize("n", [29, 30, 31])
def test_widest_boards(orc, layout, n):
    """The widest boards the 32-bit masks allow (N = 31 leaves one pre-set high
    column): seeded random prefixes eight rows short of the bottom, counts and
    nodes per prefix against the oracle."""
    d = n - 8
    q = random_placements(n, d, 1536, 3100 + n)
    cols = np.array(q, dtype=np.int8)
    want, want_n = orc.count_prefixes(n, cols)
    got, got_n, tot = run(records_of(n, q), d, n, layout, nodes=True)
    assert np.array_equal(got, want) and np.array_equal(got_n, want_n)
    assert int(tot[n]) == int(want.sum())


def test_malformed_records_are_rejected():
    pre = nq.enumerate_prefixes(10, 3).copy()
    pre["meta"][5] = (pre["meta"][5] & ~np.uint32(3))          # weight 0
    pre["cols"][7] |= np.uint32(1 << 12)                         # column outside the board
    got, _, tot = run(pre[:0], 3, 10)                           # empty: nothing recorded
    dp = nq.to_device(pre)
    cnt = torch.full((len(pre),), -1, dtype=torch.int64, device="cuda")
    nq.count(10, 3, dp, cnt)
    with pytest.raises(nq.NQError) as e:
        nq.sync()
    assert e.value.code == nq.NQ_EINVAL
    c = u64(cnt)
    assert c[5] == 0 and c[7] == 0
    nq.sync()  # the status was cleared


def test_status_belongs_to_the_stream():
    """Two streams, one of them given a malformed record: only that stream's
    nq_sync reports it; the other stream's counts and sync are clean, and a
    synchronous call in between is not failed by the pending error."""
    good = nq.enumerate_prefixes(11, 3)
    bad = good.copy()
    bad["meta"][2] = bad["meta"][2] & ~np.uint32(3)           # weight 0
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    dg, db = nq.to_device(good), nq.to_device(bad)
    cg = torch.zeros(len(good), dtype=torch.int64, device="cuda")
    cb = torch.zeros(len(bad), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    nq.count(11, 3, db, cb, stream=sb)
    nq.count(11, 3, dg, cg, stream=sa)
    assert nq.total(10) == Q[10]                  # synchronous: its own status word
    nq.sync(sa)                                   # clean
    assert int((u64(cg).astype(object) * (good["meta"] & 3).astype(object)).sum()) == Q[11]
    with pytest.raises(nq.NQError) as e:
        nq.sync(sb)
    assert e.value.code == nq.NQ_EINVAL
    nq.sync(sb)                                   # collected and cleared
    nq.sync(sa)


def test_wrong_board_size_is_rejected():
    pre = nq.enumerate_prefixes(10, 3)
    dp = nq.to_device(pre)
    cnt = torch.zeros(len(pre), dtype=torch.int64, device="cuda")
    nq.count(11, 3, dp, cnt)
    with pytest.raises(nq.NQError) as e:
        nq.sync()
    assert e.value.code == nq.NQ_EINVAL and int(cnt.abs().sum()) == 0


def test_prefix_shallower_than_declared_is_rejected():
    pre = nq.enumerate_prefixes(12, 2)
    dp = nq.to_device(pre)
    cnt = torch.zeros(len(pre), dtype=torch.int64, device="cuda")
    nq.count(12, 5, dp, cnt)          # the stack is sized for depth >= 5
    with pytest.raises(nq.NQError) as e:
        nq.sync()
    assert e.value.code == nq.NQ_ESTACK


def test_misaligned_pointer_rejected():
    pre = nq.enumerate_prefixes(10, 3)
    raw = torch.zeros(len(pre) * 4 + 1, dtype=torch.int32, device="cuda")
    mis = raw[1:].view(-1, 4)
    cnt = torch.zeros(len(pre), dtype=torch.int64, device="cuda")
    with pytest.raises(nq.NQError) as e:
        nq.count(10, 3, mis, cnt)
    assert e.value.code == nq.NQ_EINVAL


@pytest.mark.parametrize("seed", range(4))
def test_constrained_against_oracle(orc, seed):
    g = synth_inputs.SplitMix64(300 + seed)
    for _ in range(10):
        n = 4 + g.below(11)        # 4..14
        qs = synth_inputs.constraint_set(g, n, g.below(5))
        assert nq.count_constrained(n, qs) == orc.count_constrained(n, qs)[0], (n, qs)


def test_constrained_special_cases(orc):
    for n in range(1, 13):
        assert nq.count_constrained(n, []) == Q[n]
    assert nq.count_constrained(8, [(0, 0), (1, 1)]) == 0
    assert nq.count_constrained(8, [(0, 0), (0, 3)]) == 0
    assert nq.count_constrained(8, [(3, 3), (3, 3)]) == orc.count_constrained(8, [(3, 3)])[0]
    assert nq.count_constrained(9, [(8, 4)]) == orc.count_constrained(9, [(8, 4)])[0]
    assert nq.count_constrained(16, [(15, 2), (0, 7)]) == orc.count_constrained(16, [(15, 2), (0, 7)])[0]
    with pytest.raises(nq.NQError):
        nq.count_constrained(8, [(8, 1)])


@pytest.mark.slow
def test_total_n21_streamed():
    """nq_total streams N=21's 37.8 M subproblems in pieces into the running search."""
    assert nq.total(21) == Q[21]


@pytest.mark.parametrize("layout", ["regm", "reg"])
@pytest.mark.parametrize("n,d", [(16, 2), (15, 1), (17, 4), (14, 0)])
def test_subtree_donation(orc, layout, n, d):
    """Few heavy prefixes: nearly every lane starts idle and the work spreads by
    donation. Per-prefix counts and nodes equal the oracle's and the run with
    donation switched off."""
    pre = nq.enumerate_prefixes(n, d)
    want_c, want_n = oracle_counts(orc, n, d)
    for donate in (2, 1):
        got_c, got_n, tot = run(pre, d, n, layout, nodes=True, donate=donate)
        assert np.array_equal(got_c, want_c), donate
        assert np.array_equal(got_n, want_n), donate
        assert int(tot[n]) == Q[n]
        got_c2, _, tot2 = run(pre, d, n, layout, donate=donate)
        assert np.array_equal(got_c2, want_c) and int(tot2[n]) == Q[n]


def test_nodes_at_bench_depth_equal_oracle_by_refinement():
    """N=18 at d=7: the node total of the diagnostic kernel equals the oracle's
    d=5 node total minus the placements of rows 5 and 6 (the d=6 and d=7 prefix
    counts), so the bench's node count is pinned by the oracle."""
    g = np.load(os.path.join(GOLDEN, "oracle_n18_d5.npz"))
    r = nq.total_ex(18, nq.make_config(d=7), nodes=True)
    assert r["total"] == Q[18]
    assert r["nodes"] == int(g["nodes"].sum()) - nq.prefix_count(18, 6) - nq.prefix_count(18, 7)


@pytest.mark.parametrize("layout", ["regm", "reg", "wt"])
@pytest.mark.parametrize("n,d,rows", [(16, 2, 3), (15, 1, 4), (13, 4, -1), (12, 0, 5),
                                      (10, 6, 9), (9, 9, 2)])
def test_host_split_equals_oracle(orc, layout, n, d, rows):
    """nq_count_split: each prefix is expanded `rows` rows on the host and the
    children's counts and nodes are added into the parent's entry. Per-prefix
    counts and nodes equal the oracle's; rows past the last row are capped
    (d = N: the prefixes are solutions)."""
    pre = nq.enumerate_prefixes(n, d)
    want_c, want_n = oracle_counts(orc, n, d)
    r = nq.count_split(pre, rows, nq.make_config(layout), nodes=True)
    assert np.array_equal(r["counts"], want_c)
    assert np.array_equal(r["nodes"], want_n)
    assert int(r["totals"][n]) == Q[n]
    r2 = nq.count_split(pre, rows, nq.make_config(layout))
    assert np.array_equal(r2["counts"], want_c) and int(r2["totals"][n]) == Q[n]
    if rows >= 0:
        assert r["rows"] == rows


def test_host_split_golden_and_mixed(orc):
    """N=16 at d=5 against the stored oracle counts and nodes (auto rows), and
    N=10..14 mixed and shuffled in one split call."""
    g = np.load(os.path.join(GOLDEN, "oracle_n16_d5.npz"))
    r = nq.count_split(nq.enumerate_prefixes(16, 5), -1, nodes=True)
    assert np.array_equal(r["counts"], g["counts"]) and np.array_equal(r["nodes"], g["nodes"])
    assert int(r["totals"][16]) == Q[16]
    parts, want = [], []
    for n in range(10, 15):
        parts.append(nq.enumerate_prefixes(n, 2))
        want.append(oracle_counts(orc, n, 2)[0])
    pre = np.concatenate(parts)
    perm = np.random.default_rng(11).permutation(len(pre))
    r = nq.count_split(pre[perm], 3)
    assert np.array_equal(r["counts"], np.concatenate(want)[perm])
    for n in range(10, 15):
        assert int(r["totals"][n]) == Q[n]


def test_host_split_rejects_bad_input():
    pre = nq.enumerate_prefixes(10, 3).copy()
    pre["meta"][4] = (pre["meta"][4] & ~np.uint32(3)) | np.uint32(3)    # weight 3
    with pytest.raises(nq.NQError):
        nq.count_split(pre, 2)
    r = nq.count_split(pre[:0], 2)
    assert len(r["counts"]) == 0 and int(r["totals"].sum()) == 0


def test_split_word_layouts_need_256_thread_blocks():
    pre = nq.enumerate_prefixes(10, 3)
    dp = nq.to_device(pre)
    cnt = torch.zeros(len(pre), dtype=torch.int64, device="cuda")
    for layout in sorted(SPLIT_WORDS):
        with pytest.raises(nq.NQError) as e:
            nq.count_ex(dp, 3, 10, cnt, None, None, nq.make_config(layout, 128))
        assert e.value.code == nq.NQ_EINVAL


@pytest.mark.parametrize("layout", ["regp", "regz", "regpz"])
def test_streamed_total_new_layouts(layout):
    """nq_total_ex streams N=18's d=7 set (7.4 M records) into the running search
    in every register-top layout."""
    r = nq.total_ex(18, nq.make_config(layout, d=7))
    assert r["total"] == Q[18] and r["layout"] == nq.LAYOUTS[layout]


def test_avail_only_stack_limits():
    """AVAIL keeps two guard columns in its 32-bit masks: N <= 30."""
    pre = nq.prefixes_at_ranks(31, 2, [0, 1, 2, 3])
    dp = nq.to_device(pre)
    cnt = torch.zeros(len(pre), dtype=torch.int64, device="cuda")
    with pytest.raises(nq.NQError) as e:
        nq.count_ex(dp, 2, 31, cnt, None, None, nq.make_config("avail"))
    assert e.value.code == nq.NQ_EINVAL
