"""Served mode: a persistent kernel fed through a device ring (continuous
batching). Every answer is an exact integer, so the bar is equality: with the
CPU oracle, with the standalone constrained count (the same request alone),
and with OEIS for unconstrained boards."""
import json
import os
import time

import pytest

import synth_inputs
from paper_2511_12009_gb300 import nq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = {int(k): v for k, v in json.load(open(os.path.join(GOLDEN, "oeis_a000170.json")))["Q"].items()}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_stream_matches_oracle_and_standalone(orc):
    from paper_2511_12009_gb300.serve import Server, run_stream
    reqs = synth_inputs.request_stream(5, 300, 6, 14, 0, 4, rate_per_s=3000.0)
    with Server(max_n=20, request_slots=32, idle_ms=100) as srv:
        res = run_stream(srv, reqs, timeout_s=300)
        st = srv.stats()
    assert st["submitted"] == st["completed"] == len(reqs)
    for i, r in enumerate(reqs):
        want = orc.count_constrained(r["n"], r["queens"])[0]
        assert res["answers"][i] == want, (r["n"], r["queens"])
        if i % 10 == 0:
            assert nq.count_constrained(r["n"], r["queens"]) == want


@pytest.mark.parametrize("max_n,slots", [(16, 6), (17, 12), (20, 12)])
def test_largest_boards_at_the_stack_limit(orc, max_n, slots):
    """Requests at the server's largest board size, where the depth the stack
    footprint forces (N - 1 - d frames) decides whether a record fits: answers
    against the standalone count and, for small boards, the oracle; boards
    without queens against OEIS."""
    from paper_2511_12009_gb300.serve import Server, run_stream
    g = synth_inputs.SplitMix64(4000 + max_n)
    reqs = []
    for i in range(12):
        k = [0, 1, 2][i % 3]
        reqs.append({"id": i, "t": 0.0, "n": max_n,
                     "queens": synth_inputs.constraint_set(g, max_n, k)})
    with Server(max_n=max_n, stack_slots=slots, request_slots=16, idle_ms=100) as srv:
        res = run_stream(srv, reqs, timeout_s=600)
        assert srv.poll() == []      # no error surfaced after the last answer
    for i, r in enumerate(reqs):
        if not r["queens"]:
            assert res["answers"][i] == Q[max_n]
        else:
            want = nq.count_constrained(max_n, r["queens"])
            assert res["answers"][i] == want, (r["queens"],)
            if max_n <= 16:
                assert want == orc.count_constrained(max_n, r["queens"])[0]


def test_light_requests_overtake_a_heavy_one():
    from paper_2511_12009_gb300.serve import Server
    with Server(max_n=20, request_slots=64, idle_ms=200) as srv:
        heavy = srv.submit(19, [])
        light = [srv.submit(11, [(0, c)]) for c in range(5)]
        assert heavy is not None and None not in light
        order, answers = [], {}
        t0 = time.time()
        while len(answers) < 6 and time.time() - t0 < 120:
            for t, c in srv.poll():
                order.append(t)
                answers[t] = c
            time.sleep(1e-4)
    assert answers[heavy] == Q[19]
    # the light requests were admitted while the heavy one ran and finished first
    assert order.index(heavy) == len(order) - 1
    for j, t in enumerate(light):
        assert answers[t] == nq.count_constrained(11, [(0, j)])


def test_idle_exit_and_relaunch():
    from paper_2511_12009_gb300.serve import Server
    with Server(max_n=16, request_slots=8, idle_ms=5) as srv:
        a = srv.submit(12, [(3, 4)])
        got = {}
        while a not in got:
            got.update(dict(srv.poll()))
        time.sleep(0.5)            # longer than the idle limit: the kernel leaves
        b = srv.submit(12, [(5, 1)])
        while b not in got:
            got.update(dict(srv.poll()))
        st = srv.stats()
    assert got[a] == nq.count_constrained(12, [(3, 4)])
    assert got[b] == nq.count_constrained(12, [(5, 1)])
    assert st["launches"] >= 2


def test_admission_refuses_when_full():
    from paper_2511_12009_gb300.serve import Server
    with Server(max_n=20, request_slots=2, idle_ms=200) as srv:
        t1 = srv.submit(18, [])
        t2 = srv.submit(18, [(0, 1)])
        t3 = srv.submit(17, [])
        assert t1 is not None and t2 is not None and t3 is None
        got = {}
        while len(got) < 2:
            got.update(dict(srv.poll()))
        t3 = srv.submit(17, [])
        while t3 not in got:
            got.update(dict(srv.poll()))
    assert got[t1] == Q[18] and got[t3] == Q[17]
    assert got[t2] == nq.count_constrained(18, [(0, 1)])


def test_conflicting_and_invalid_requests():
    from paper_2511_12009_gb300.serve import Server
    with Server(max_n=16, request_slots=4, idle_ms=50) as srv:
        t = srv.submit(10, [(0, 0), (1, 1)])
        got = {}
        while t not in got:
            got.update(dict(srv.poll()))
        assert got[t] == 0
        with pytest.raises(nq.NQError):
            srv.submit(17, [])          # above the server's max_n
        with pytest.raises(nq.NQError):
            srv.submit(10, [(10, 0)])   # off the board


@pytest.mark.parametrize("seed", [1, 2])
def test_board_symmetry_served(seed):
    """count(Q) = count(g.Q) for the 8 symmetries of the square, on N = 16..18."""
    from paper_2511_12009_gb300.serve import Server
    g = synth_inputs.SplitMix64(900 + seed)
    n = 16 + g.below(3)
    qs = synth_inputs.constraint_set(g, n, 2)
    f = n - 1
    maps = [lambda r, c: (r, c), lambda r, c: (c, f - r), lambda r, c: (f - r, f - c),
            lambda r, c: (f - c, r), lambda r, c: (r, f - c), lambda r, c: (f - r, c),
            lambda r, c: (c, r), lambda r, c: (f - c, f - r)]
    with Server(max_n=18, request_slots=16, idle_ms=100) as srv:
        tickets = [srv.submit(n, [m(r, c) for r, c in qs]) for m in maps]
        got = {}
        while len(got) < len(tickets):
            got.update(dict(srv.poll()))
    vals = {got[t] for t in tickets}
    assert len(vals) == 1
    assert vals.pop() == nq.count_constrained(n, qs)
