"""GPU parity on the paper's larger boards (Tables 3-6 run N = 17..22).

Every per-prefix solution count and node count of the CUDA search is compared,
element by element, with arrays the CPU oracle wrote (tests/golden/
make_golden.py, which calls only oracle/):
  - N = 19, all 232,174 prefixes of depth 5, in the default layout and in REG;
  - N = 20, 21, 22: 2,048 seeded prefixes each at the library's depth 7,
    counted in a launch of their own, and the same indices read out of a full
    count of the whole board in the default launch (the configuration the
    benchmark times), whose weighted total must equal Q(N).
Counts are integers: the bar is exact equality.
"""
import json
import os

import numpy as np
import pytest

from paper_2511_12009_gb300 import nq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = {int(k): v for k, v in json.load(open(os.path.join(GOLDEN, "oeis_a000170.json")))["Q"].items()}
SAMPLED = {20: "oracle_n20_d7_s2048.npz", 21: "oracle_n21_d7_s2048.npz",
           22: "oracle_n22_d7_s2048.npz"}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nq.lib()


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def search(pre, min_d, max_n, layout="default", nodes=False):
    dp = nq.to_device(pre)
    m = len(pre)
    cnt = torch.full((max(m, 1),), -1, dtype=torch.int64, device="cuda")
    nod = torch.full((max(m, 1),), -1, dtype=torch.int64, device="cuda") if nodes else None
    tot = torch.zeros(32, dtype=torch.int64, device="cuda")
    nq.count_ex(dp, min_d, max_n, cnt, nod, tot, nq.make_config(layout))
    nq.sync()
    return u64(cnt)[:m], (u64(nod)[:m] if nodes else None), u64(tot)


@pytest.mark.parametrize("layout", ["default", "reg"])
def test_n19_every_prefix(layout):
    g = np.load(os.path.join(GOLDEN, "oracle_n19_d5.npz"))
    pre = nq.enumerate_prefixes(19, 5)
    assert len(pre) == len(g["counts"]) == 232174
    assert np.array_equal(pre["meta"] & 3, g["weights"])
    got_c, got_n, tot = search(pre, 5, 19, layout, nodes=True)
    assert np.array_equal(got_c, g["counts"])
    assert np.array_equal(got_n, g["nodes"])
    assert int(tot[19]) == Q[19]
    got_c2, _, tot2 = search(pre, 5, 19, layout)  # production build: no node counters
    assert np.array_equal(got_c2, g["counts"]) and int(tot2[19]) == Q[19]


@pytest.mark.parametrize("n", [20, 21, 22])
def test_sampled_prefixes_own_launch(n):
    """The seeded sample alone: counts from the production kernel, counts and
    nodes from the diagnostic build, each against the oracle's arrays."""
    g = np.load(os.path.join(GOLDEN, SAMPLED[n]))
    d = 7
    assert nq.prefix_count(n, d) == int(g["set_size"][0])
    pre = nq.prefixes_at_ranks(n, d, g["ranks"])
    assert np.array_equal(pre["meta"] & 3, g["weights"])
    got_c, _, tot = search(pre, d, n)
    assert np.array_equal(got_c, g["counts"])
    assert int(tot[n]) == int((g["weights"].astype(np.uint64) * g["counts"]).sum())
    got_c2, got_n, _ = search(pre, d, n, "regm", nodes=True)
    assert np.array_equal(got_c2, g["counts"])
    assert np.array_equal(got_n, g["nodes"])


@pytest.mark.slow
@pytest.mark.parametrize("n", [20, 21, 22])
def test_full_board_sampled_outputs(n):
    """The whole depth-7 set of the board in the default launch (the
    benchmark's configuration): the sampled entries of the per-prefix output
    equal the oracle's, and the weighted total equals Q(N)."""
    g = np.load(os.path.join(GOLDEN, SAMPLED[n]))
    pre = nq.enumerate_prefixes(n, 7)
    assert len(pre) == int(g["set_size"][0])
    dp = nq.to_device(pre)
    del pre
    cnt = torch.full((dp.shape[0],), -1, dtype=torch.int64, device="cuda")
    tot = torch.zeros(32, dtype=torch.int64, device="cuda")
    nq.count_ex(dp, 7, n, cnt, None, tot, None)
    nq.sync()
    del dp
    idx = torch.from_numpy(g["ranks"].astype(np.int64)).cuda()
    assert np.array_equal(u64(cnt[idx]), g["counts"])
    assert int(u64(tot)[n]) == Q[n]
