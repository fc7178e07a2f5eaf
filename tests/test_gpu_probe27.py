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
