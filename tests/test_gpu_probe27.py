"""N=27 scale probe: 4096 seeded subtrees of the 27-Queens problem.

Sample: ranks drawn uniformly (SplitMix64, seed 27) over the canonical depth-8
prefix set, each prefix then extended two rows by a seeded choice among its
depth-10 descendants (index = draw mod count; a prefix with none is skipped
and the next rank taken). Depth 10 keeps each subtree near a few CPU-core
seconds of oracle work. The GPU counts all 4096; the oracle, with its own
unranking and its own descendant enumeration, re-derives the first 256
prefixes and counts them one by one; the host-split call must give the
same 4096 counts. Exact equality throughout.
"""
import numpy as np
import pytest

import synth_inputs
from paper_2511_12009_gb300 import nq

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

N, D0, EXTRA, K, CHECK = 27, 8, 2, 4096, 256


def to_state(n, cols_list):
    d = len(cols_list)
    cols = sum(1 << int(c) for c in cols_list)
    ld = sum(1 << (int(c) + d - r) for r, c in enumerate(cols_list) if int(c) + d - r < n)
    rd = sum(1 << (int(c) - d + r) for r, c in enumerate(cols_list) if int(c) - d + r >= 0)
    return cols, ld, rd


@pytest.fixture(scope="module")
def sample():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    total = nq.prefix_count(N, D0)
    ranks = synth_inputs.sample_ranks(27, total, K + 256)
    choices = synth_inputs.raw_u64(2700, K + 256)
    parents = nq.prefixes_at_ranks(N, D0, ranks)
    picked, used = [], []
    for i, p in enumerate(parents):
        kids = nq.descendants(p, EXTRA)
        if len(kids) == 0:
            continue
        picked.append(kids[choices[i] % len(kids)])
        used.append(i)
        if len(picked) == K:
            break
    assert len(picked) == K
    return ranks, choices, np.array(picked, dtype=nq.PREFIX_DTYPE), used


def test_probe_counts_against_oracle(orc, sample):
    ranks, choices, pre, used = sample
    dp = nq.to_device(pre)
    cnt = torch.zeros(K, dtype=torch.int64, device="cuda")
    nq.count(N, D0 + EXTRA, dp, cnt)
    nq.sync()
    got = cnt.cpu().numpy().view(np.uint64)
    assert int(got.sum()) > 0
    # oracle: its own unranking and descendant enumeration for the first CHECK
    idx = used[:CHECK]
    parents = orc.prefixes_at_ranks(N, D0, [ranks[i] for i in idx])
    oracle_cols = []
    for j, i in enumerate(idx):
        kids = orc.descendants(N, parents[j], EXTRA)
        oracle_cols.append(kids[choices[i] % len(kids)])
    for j, cl in enumerate(oracle_cols):
        rec = pre[j]
        assert (int(rec["cols"]), int(rec["ld"]), int(rec["rd"])) == to_state(N, cl)
    want, _ = orc.count_prefixes(N, np.array(oracle_cols, dtype=np.int8))
    assert np.array_equal(got[:CHECK], want)
    # the host split (children searched in one launch, summed per parent) agrees
    split = nq.count_split(pre, -1)
    assert split["rows"] >= 1
    assert np.array_equal(split["counts"], got)


class _Stop(Exception):
    pass


def big_sample(k, seed_ranks=2727, seed_choice=27270):
    """k seeded depth-10 subtrees of the 27-Queens problem, by the probe's recipe
    (uniform ranks at depth 8, a seeded choice among each prefix's depth-10
    descendants), with their parents' ranks and the choices made."""
    total = nq.prefix_count(N, D0)
    ranks = synth_inputs.sample_ranks(seed_ranks, total, k + k // 8)
    choices = synth_inputs.raw_u64(seed_choice, k + k // 8)
    picked, used = [], []
    for i, p in enumerate(nq.prefixes_at_ranks(N, D0, ranks)):
        kids = nq.descendants(p, EXTRA)
        if len(kids):
            picked.append(kids[choices[i] % len(kids)])
            used.append(i)
        if len(picked) == k:
            break
    assert len(picked) == k
    return ranks, choices, np.array(picked, dtype=nq.PREFIX_DTYPE), used


def test_long_run_through_the_checkpointing_driver(orc, tmp_path):
    """65,536 seeded N=27 subtrees through shard.count_board with a checkpoint:
    stopped on the host after three pieces, resumed with another piece size.
    Every subtree is counted exactly once; all counts equal a separate count of
    the whole sample in one host-split call, and the first 256 equal the
    oracle's (its own unranking, descendant choice and backtracker)."""
    from paper_2511_12009_gb300 import shard
    k = 65536
    ranks, choices, pre, used = big_sample(k)
    ck = str(tmp_path / "n27")
    counter = shard.gpu_counter(split=True)
    seen = []

    def stop_after_three(lo, hi):
        seen.append((lo, hi))
        if len(seen) == 3:
            raise _Stop()

    with pytest.raises(_Stop):
        shard.count_board(N, records=pre, chunk=8192, counter=counter, checkpoint=ck,
                          on_piece=stop_after_three)
    r = shard.count_board(N, records=pre, chunk=6000, counter=counter, checkpoint=ck)
    assert r["resumed"] == 3 * 8192 and r["records"] == k
    header = {"n": N, "d": D0 + EXTRA, "records": k, "sample": shard.records_digest(pre)}
    got = np.zeros(k, dtype=np.uint64)
    times = np.zeros(k, dtype=np.int64)
    for lo, c in shard.read_checkpoint(ck, header).items():
        got[lo:lo + len(c)] = c
        times[lo:lo + len(c)] += 1
    assert (times == 1).all()                    # every subtree exactly once
    whole = nq.count_split(pre, -1)["counts"]
    assert np.array_equal(got, whole)
    assert r["total"] == int((got.astype(object) * 2).sum())  # every weight is 2
    idx = used[:CHECK]
    parents = orc.prefixes_at_ranks(N, D0, [ranks[i] for i in idx])
    cols = []
    for j, i in enumerate(idx):
        kids = orc.descendants(N, parents[j], EXTRA)
        cols.append(kids[choices[i] % len(kids)])
    want, _ = orc.count_prefixes(N, np.array(cols, dtype=np.int8))
    assert np.array_equal(got[:CHECK], want)
