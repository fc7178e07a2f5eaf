"""The multi-worker driver on the GPU (one worker here): libnq's search kernel
as the counter, a run stopped between pieces on the host, then resumed from
its checkpoint log. Per-prefix counts are compared with the oracle's stored
arrays (tests/golden, written by make_golden.py from oracle/ only)."""
import json
import os

import numpy as np
import pytest

from paper_2511_12009_gb300 import nq, shard

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nq.lib()


class Stop(Exception):
    pass


@pytest.mark.parametrize("mode", ["lease", "static"])
def test_gpu_counter_checkpoint_resume(tmp_path, mode):
    n, d = 16, 5
    z = np.load(os.path.join(GOLDEN, f"oracle_n{n}_d{d}.npz"))
    q = json.load(open(os.path.join(GOLDEN, "oeis_a000170.json")))["Q"][str(n)]
    ck = str(tmp_path / "ck")
    seen = []

    def stop_after_three(lo, hi):
        seen.append((lo, hi))
        if len(seen) == 3:
            raise Stop()

    with pytest.raises(Stop):
        shard.count_board(n, d, mode=mode, chunk=7001, checkpoint=ck, on_piece=stop_after_three)
    counts = np.zeros(len(z["counts"]), dtype=np.uint64)
    got = np.zeros(len(counts), dtype=bool)
    done = shard.read_checkpoint(ck, {"n": n, "d": d, "records": len(counts)})
    assert done.covered() == 3 * 7001
    for lo, c in done.items():
        counts[lo:lo + len(c)] = c
        got[lo:lo + len(c)] = True
    r = shard.count_board(n, d, mode=mode, chunk=5000, checkpoint=ck)
    assert r["total"] == q
    for lo, c in r["pieces"].items():
        assert not got[lo:lo + len(c)].any()  # nothing counted twice
        counts[lo:lo + len(c)] = c
        got[lo:lo + len(c)] = True
    assert got.all()
    assert np.array_equal(counts, z["counts"])


def test_gpu_static_ratio_slices_sum_to_the_total():
    """Eight workers' static ratio slices (Section 4.5), run one after another
    on this GPU, add up to Q(N); each slice's counts match the oracle's."""
    n, d = 17, 5
    z = np.load(os.path.join(GOLDEN, f"oracle_n{n}_d{d}.npz"))
    q = json.load(open(os.path.join(GOLDEN, "oeis_a000170.json")))["Q"][str(n)]
    ratios = [0.20, 0.15, 0.12, 0.11, 0.11, 0.11, 0.10, 0.10]
    total = 0
    for rank in range(8):
        r = shard.count_board(n, d, rank=rank, world=8, mode="static", ratios=ratios,
                              chunk=1 << 20)
        total += r["total"]
        for lo, c in r["pieces"].items():
            assert np.array_equal(c, z["counts"][lo:lo + len(c)])
    assert total == q
