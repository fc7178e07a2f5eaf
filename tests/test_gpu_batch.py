"""Batched counting (one persistent launch over several board sizes, replayed
from a CUDA graph), work-chunk claiming and the autotuner: every answer is the
exact count, the same batched and alone."""
import json
import os

import numpy as np
import pytest

from paper_2511_12009_gb300 import nq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = {int(k): v for k, v in json.load(open(os.path.join(GOLDEN, "oeis_a000170.json")))["Q"].items()}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_batch_small_boards_per_prefix(orc):
    from paper_2511_12009_gb300.batch import Batch
    ns = [14, 9, 11, 8, 13, 10, 12]          # unsorted on purpose
    ds = [5, 3, 0, 2, 4, 3, 0]
    with Batch(ns, ds) as b:
        info = b.info()
        assert info["max_n"] == 14 and info["min_d"] == 2
        tot, ms = b.run()
        assert tot == [Q[n] for n in ns] and ms > 0
        for i, n in enumerate(ns):
            d = ds[i] or nq.default_depth(n)
            want, _ = orc.count_prefixes(n, orc.prefixes(n, d)[0])
            assert np.array_equal(b.counts(i), want), n
        tot2, _ = b.run()                       # graph replay again
        assert tot2 == tot
        tot3, _ = b.run_separate()
        assert tot3 == tot
        for i, n in enumerate(ns):              # per-prefix counts of the separate run
            d = ds[i] or nq.default_depth(n)
            want, _ = orc.count_prefixes(n, orc.prefixes(n, d)[0])
            assert np.array_equal(b.counts(i), want), n


@pytest.mark.parametrize("layout", ["regm", "reg", "paper"])
def test_batch_larger_boards(layout):
    from paper_2511_12009_gb300.batch import Batch
    ns = [15, 16, 17, 18]
    with Batch(ns, None, nq.make_config(layout, claim=2)) as b:
        tot, _ = b.run()
        assert tot == [Q[n] for n in ns]
        tot2, _ = b.run_separate()
        assert tot2 == tot


def test_batch_rejects_duplicates_and_overflow():
    from paper_2511_12009_gb300.batch import Batch
    with pytest.raises(nq.NQError):
        Batch([10, 10])
    with pytest.raises(nq.NQError):
        Batch([29])


@pytest.mark.parametrize("claim", [1, 2, 5, 16, 64])
def test_claim_chunks_keep_counts(orc, claim):
    n, d = 13, 5
    pre = nq.enumerate_prefixes(n, d)
    want, _ = orc.count_prefixes(n, orc.prefixes(n, d)[0])
    for layout in ("regm", "reg", "wt"):
        dp = nq.to_device(pre)
        cnt = torch.zeros(len(pre), dtype=torch.int64, device="cuda")
        tot = torch.zeros(32, dtype=torch.int64, device="cuda")
        nq.count_ex(dp, d, n, cnt, None, tot, nq.make_config(layout, claim=claim))
        nq.sync()
        assert np.array_equal(cnt.cpu().numpy().view(np.uint64), want)
        assert int(tot[n]) == Q[n]


def test_tuner_finds_a_correct_config(tmp_path, monkeypatch):
    from paper_2511_12009_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune.json"))
    cfg = tune.tune(13, reps=1, layouts=("regm", "reg"), blocks=(128, 256), claims=(1, 4))
    assert tune.cached(13) == cfg
    r = nq.total_ex(13, tune.best_config(13))
    assert r["total"] == Q[13]
    rec = tune.tune_batch([10, 11, 12], reps=1, blocks=(128,), claims=(1,))
    assert rec["totals"] == [Q[10], Q[11], Q[12]]


def test_separate_launches_after_planning_every_board():
    """Planning several boards, then launching them: the board planned last
    (N=15 at depth 1: 15 frames, the planner picks 224-thread blocks) needs less
    shared memory per block than one planned before it (N=14 at depth 1: 14
    frames, 256-thread blocks). Every launch must still be valid."""
    from paper_2511_12009_gb300.batch import Batch
    with Batch([14, 15], [1, 1], None) as b:
        totals, _ = b.run()
        sep, _ = b.run_separate()
    assert totals == sep == [Q[14], Q[15]]
