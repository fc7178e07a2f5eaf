"""CPU tests of two host-side drivers whose GPU work is stubbed out: the
autotuner's staged search and cache (`tune.py`), and the served-stream replay
(`serve.run_stream`: arrivals, refusals while the server is full, completion
and latency bookkeeping). The stubs stand in for libnq calls only; the search
itself is covered by the GPU tests."""
import json

import pytest

from paper_2511_12009_gb300 import nq, tune
from paper_2511_12009_gb300.serve import run_stream


# --- autotuner ---------------------------------------------------------------

class FakeTotalEx:
    """nq_total_ex stand-in: a made-up cost per configuration, the right total."""

    def __init__(self, cost, total=14200, wrong=None):
        self.cost, self.total, self.wrong, self.calls = cost, total, wrong, []

    def __call__(self, n, config=None, nodes=False):
        cfg = {f: getattr(config, f) for f in ("layout", "block", "blocks_per_sm", "order", "d",
                                               "claim")}
        self.calls.append(cfg)
        bad = self.wrong is not None and self.wrong(cfg)
        return {"total": self.total + (1 if bad else 0), "kernel_ms": self.cost(cfg)}


@pytest.fixture
def tuner(monkeypatch, tmp_path):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    monkeypatch.setattr(tune, "_device_key", lambda: "fake-gpu|152")
    return tune


def test_staged_search_keeps_the_best_of_each_stage(tuner, monkeypatch):
    d0 = nq.default_depth(12)

    def cost(c):  # depth d0 + 1 best, then layout reg, then block 128 in index order, claim 2
        ms = 10.0 - (2.0 if c["d"] == d0 + 1 else 0.0)
        ms -= 1.0 if c["layout"] == nq.LAYOUTS["reg"] else 0.0
        ms -= 0.5 if (c["block"], c["order"]) == (128, 1) else 0.0
        ms -= 0.25 if c["claim"] == 2 else 0.0
        return ms

    fake = FakeTotalEx(cost)
    monkeypatch.setattr(nq, "total_ex", fake)
    best = tuner.tune(12, reps=1)
    assert best == {"layout": nq.LAYOUTS["reg"], "block": 128, "blocks_per_sm": 0, "order": 1,
                    "d": d0 + 1, "claim": 2}
    rec = json.load(open(tuner.CACHE))["fake-gpu|152|N=12"]
    assert rec["config"] == best and rec["ms"] == pytest.approx(6.25)
    assert len(rec["tried"]) == len(fake.calls)
    assert tuner.cached(12) == best
    cfg = tuner.best_config(12)
    assert (cfg.layout, cfg.block, cfg.order, cfg.d, cfg.claim) == (best["layout"], 128, 1,
                                                                     d0 + 1, 2)


def test_a_config_with_another_total_is_an_error(tuner, monkeypatch):
    fake = FakeTotalEx(lambda c: 1.0, wrong=lambda c: c["layout"] == nq.LAYOUTS["wt"])
    monkeypatch.setattr(nq, "total_ex", fake)
    with pytest.raises(RuntimeError, match="expected"):
        tuner.tune(12, reps=1)


def test_untuned_board_gets_the_library_default(tuner):
    cfg = tuner.best_config(13)
    assert (cfg.layout, cfg.d) == (0, nq.default_depth(13))


# --- served-stream replay ---------------------------------------------------------

class FakeServer:
    """Admits at most `slots` requests at once; a request completes after
    `polls` polls; its answer is n * 1000 + number of queens."""

    def __init__(self, slots=2, polls=3):
        self.slots, self.polls = slots, polls
        self.live = {}  # ticket -> [polls left, answer]
        self.next = 1
        self.refused = 0

    def submit(self, n, queens):
        if len(self.live) >= self.slots:
            self.refused += 1
            return None
        t = self.next
        self.next += 1
        self.live[t] = [self.polls, n * 1000 + len(queens)]
        return t

    def poll(self):
        out = []
        for t in list(self.live):
            self.live[t][0] -= 1
            if self.live[t][0] <= 0:
                out.append((t, self.live.pop(t)[1]))
        return out


def test_stream_replay_answers_every_request_once():
    reqs = [{"t": 0.0, "n": 10 + i % 5, "queens": [(0, j) for j in range(i % 3)]}
            for i in range(12)]
    srv = FakeServer(slots=2, polls=3)
    res = run_stream(srv, reqs, timeout_s=30)
    assert res["answers"] == {i: r["n"] * 1000 + len(r["queens"]) for i, r in enumerate(reqs)}
    assert set(res["latency_s"]) == set(range(len(reqs)))
    assert all(v >= 0 for v in res["latency_s"].values())
    assert res["busy_retries"] == srv.refused > 0  # two slots for twelve requests


def test_stream_replay_waits_for_arrivals():
    reqs = [{"t": 0.05 * i, "n": 8, "queens": []} for i in range(4)]
    res = run_stream(FakeServer(slots=8, polls=1), reqs, timeout_s=30)
    assert len(res["answers"]) == 4 and res["wall_s"] >= 0.15


def test_stream_replay_times_out():
    class Stuck(FakeServer):
        def poll(self):
            return []
    with pytest.raises(TimeoutError):
        run_stream(Stuck(), [{"t": 0.0, "n": 8, "queens": []}], timeout_s=0.2)
