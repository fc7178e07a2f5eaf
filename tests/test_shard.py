"""Multi-worker counting (Section 4.5) on the CPU: gloo ranks, world size 2.

The workers' counting step is the oracle here (each worker maps its records to
the oracle's column lists by canonical index), so these tests cover the host
logic -- the static and leased splits, the final sum, checkpoint / resume and
a worker that fails between pieces -- with no GPU. Failures are made on the
host: a worker raises, the survivor's collective ends with an error.
"""
import datetime
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2511_12009_gb300 import nq, shard  # noqa: E402

OEIS = {8: 92, 9: 352, 10: 724, 11: 2680, 12: 14200}


class OracleCounter:
    """counter(records) -> counts through the oracle, by canonical index."""

    def __init__(self, n, d):
        import oracle
        oracle.build()
        self.oracle = oracle
        self.n = n
        cols, _ = oracle.prefixes(n, d)
        recs = nq.enumerate_prefixes(n, d)
        assert len(recs) == len(cols)
        self.index = {(int(r["cols"]), int(r["ld"]), int(r["rd"])): i for i, r in enumerate(recs)}
        self.cols = cols
        self.calls = 0
        self.counted = 0

    def __call__(self, records):
        self.calls += 1
        self.counted += len(records)
        idx = [self.index[(int(r["cols"]), int(r["ld"]), int(r["rd"]))] for r in records]
        counts, _ = self.oracle.count_prefixes(self.n, self.cols[idx], threads=1)
        return counts


def _worker(rank, world, store_path, result_dir, kwargs, fail_after):
    store = dist.FileStore(store_path, world)
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    n, d = kwargs["n"], kwargs["d"]
    pieces = []

    def on_piece(lo, hi):
        pieces.append((lo, hi))
        if fail_after is not None and rank == fail_after[0] and len(pieces) >= fail_after[1]:
            raise RuntimeError("injected worker failure")

    status = "ok"
    try:
        res = shard.count_board(rank=rank, world=world, store=store,
                                counter=OracleCounter(n, d), on_piece=on_piece, **kwargs)
        out = {"total": res["total"], "local": res["local_total"],
               "pieces": {int(k): v.tolist() for k, v in res["pieces"].items()}}
    except Exception as e:  # reported to the parent, which decides what was expected
        status = f"error: {type(e).__name__}: {e}"
        out = {}
    np.save(os.path.join(result_dir, f"rank{rank}.npy"),
            np.array([{"status": status, **out}], dtype=object), allow_pickle=True)
    try:
        dist.destroy_process_group()
    except Exception:
        pass


def run_world(tmp_path, world, kwargs, fail_after=None, tag="run"):
    store_path = str(tmp_path / f"store_{tag}")
    result_dir = tmp_path / f"res_{tag}"
    result_dir.mkdir()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, store_path, str(result_dir), kwargs,
                                                fail_after)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode is not None, "worker did not finish"
    return [np.load(result_dir / f"rank{r}.npy", allow_pickle=True)[0] for r in range(world)]


@pytest.mark.parametrize("mode,ratios", [("lease", None), ("static", None),
                                         ("static", [0.7, 0.3])])
def test_two_workers_total(tmp_path, mode, ratios):
    n, d = 10, 3
    res = run_world(tmp_path, 2, {"n": n, "d": d, "mode": mode, "ratios": ratios, "chunk": 7})
    assert all(r["status"] == "ok" for r in res), res
    assert res[0]["total"] == res[1]["total"] == OEIS[n]
    assert res[0]["local"] + res[1]["local"] == OEIS[n]
    # the workers' pieces cover every subproblem once
    m = nq.prefix_count(n, d)
    cover = np.zeros(m, dtype=int)
    for r in res:
        for lo, counts in r["pieces"].items():
            cover[lo:lo + len(counts)] += 1
    assert (cover == 1).all()
    if mode == "static":
        first, cnt = nq.partition(m, 2, ratios)[1]
        assert min(res[1]["pieces"]) == first
        assert sum(len(c) for c in res[1]["pieces"].values()) == cnt


def test_failed_worker_then_resume(tmp_path):
    """Worker 1 fails after its second piece; worker 0's final sum ends with an
    error instead of waiting forever; a fresh single worker resumes from both
    logs, counts only what is missing and gets the exact total."""
    n, d, chunk = 11, 3, 9
    ck = str(tmp_path / "ckpt")
    res = run_world(tmp_path, 2, {"n": n, "d": d, "mode": "lease", "chunk": chunk,
                                  "checkpoint": ck}, fail_after=(1, 2), tag="a")
    assert res[1]["status"].startswith("error") and "injected" in res[1]["status"]
    assert res[0]["status"].startswith("error")  # the all-reduce lost its peer
    m = nq.prefix_count(n, d)
    header = {"n": n, "d": d, "records": m}
    done = shard.read_checkpoint(ck, header)
    assert 0 < done.covered() <= m
    counter = OracleCounter(n, d)
    r = shard.count_board(n, d, mode="lease", chunk=5, counter=counter, checkpoint=ck)
    assert r["total"] == OEIS[n]
    assert counter.counted == m - done.covered()
    # a second resume has nothing left to count
    counter2 = OracleCounter(n, d)
    r2 = shard.count_board(n, d, mode="static", chunk=4, counter=counter2, checkpoint=ck)
    assert r2["total"] == OEIS[n] and counter2.counted == 0


def test_resume_drops_a_torn_record(tmp_path):
    n, d = 10, 3
    ck = str(tmp_path / "ck")
    c1 = OracleCounter(n, d)
    calls = []

    def stop(lo, hi):
        calls.append(lo)
        if len(calls) == 3:
            raise KeyboardInterrupt  # the process is stopped between pieces
    with pytest.raises(KeyboardInterrupt):
        shard.count_board(n, d, mode="lease", chunk=6, counter=c1, checkpoint=ck, on_piece=stop)
    log = ck + ".rank0"
    size = os.path.getsize(log)
    with open(log, "ab") as f:  # a crash in the middle of the fourth record
        f.write(b"\x07" * 13)
    header = {"n": n, "d": d, "records": nq.prefix_count(n, d)}
    assert shard.read_checkpoint(ck, header).covered() == 18
    # damage inside the third record: it and everything after it are dropped
    with open(log, "r+b") as f:
        f.seek(size - 5)
        f.write(b"\xff")
    assert shard.read_checkpoint(ck, header).covered() == 12
    c2 = OracleCounter(n, d)
    r = shard.count_board(n, d, mode="lease", chunk=6, counter=c2, checkpoint=ck)
    assert r["total"] == OEIS[n]
    assert c2.counted == header["records"] - 12


def test_checkpoint_of_another_job_is_refused(tmp_path):
    ck = str(tmp_path / "ck")
    shard.count_board(9, 2, mode="lease", chunk=4, counter=OracleCounter(9, 2), checkpoint=ck)
    with pytest.raises(shard.CheckpointError):
        shard.count_board(9, 3, mode="lease", chunk=4, counter=OracleCounter(9, 3), checkpoint=ck)
    with open(ck + ".rank0", "r+b") as f:
        f.write(b"garbage")
    with pytest.raises(shard.CheckpointError):
        shard.read_checkpoint(ck, {"n": 9, "d": 2, "records": nq.prefix_count(9, 2)})


def test_conflicting_records_are_refused():
    done = shard.Done()
    done.add(0, np.array([1, 2, 3], dtype=np.uint64))
    done.add(2, np.array([3, 4], dtype=np.uint64))  # agrees on the shared subproblem
    assert done.covered() == 4 and done.missing(0, 6) == [(4, 6)]
    with pytest.raises(shard.CheckpointError):
        done.add(1, np.array([9], dtype=np.uint64))
    # a range spanning several recorded ones is checked against each of them
    done.add(10, np.array([7, 7], dtype=np.uint64))
    done.add(20, np.array([5], dtype=np.uint64))
    with pytest.raises(shard.CheckpointError):  # agrees at 3 and 10..11, not at 20
        done.add(3, np.array([4] + [0] * 6 + [7, 7] + [0] * 8 + [6], dtype=np.uint64))
    assert done.missing(0, 22) == [(4, 10), (12, 20), (21, 22)]
    done.add(3, np.array([4] + [0] * 6 + [7, 7] + [0] * 8 + [5, 0], dtype=np.uint64))
    assert done.missing(0, 22) == [] and done.covered() == 22


def test_single_worker_splits_agree():
    n, d = 12, 4
    totals = set()
    for mode, chunk in [("lease", 1), ("lease", 100), ("static", 37)]:
        totals.add(shard.count_board(n, d, mode=mode, chunk=chunk,
                                     counter=OracleCounter(n, d))["total"])
    assert totals == {OEIS[n]}


def test_sample_of_records_checkpoint_and_refusal(tmp_path):
    """count_board over an explicit sample (a board too large to count whole):
    stopped between pieces, resumed with another chunk size, every record
    counted once and equal to the oracle; a log written for another sample
    is refused."""
    n, d = 11, 4
    counter = OracleCounter(n, d)
    recs = nq.enumerate_prefixes(n, d)
    pick = np.random.default_rng(3).permutation(len(recs))[:200]
    sample = recs[pick]
    want = counter(sample)
    ck = str(tmp_path / "ck")

    class Stop(Exception):
        pass

    seen = []

    def stop_after_two(lo, hi):
        seen.append((lo, hi))
        if len(seen) == 2:
            raise Stop()

    with pytest.raises(Stop):
        shard.count_board(n, records=sample, chunk=37, counter=counter, checkpoint=ck,
                          on_piece=stop_after_two)
    r = shard.count_board(n, records=sample, chunk=50, counter=counter, checkpoint=ck)
    assert r["resumed"] == 2 * 37 and r["records"] == 200
    got = np.zeros(200, dtype=np.uint64)
    covered = np.zeros(200, dtype=bool)
    for lo, c in shard.read_checkpoint(ck, {"n": n, "d": d, "records": 200,
                                            "sample": shard.records_digest(sample)}).items():
        got[lo:lo + len(c)] = c
        covered[lo:lo + len(c)] = True
    assert covered.all() and np.array_equal(got, want)
    assert r["total"] == int(sum(int(m & 3) * int(c) for m, c in zip(sample["meta"], want)))
    with pytest.raises(shard.CheckpointError):
        shard.count_board(n, records=sample[::-1].copy(), chunk=50, counter=counter,
                          checkpoint=ck)
