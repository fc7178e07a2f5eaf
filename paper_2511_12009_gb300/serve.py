"""Request server (binding of the nq_server_* calls) and a driver for a
timed request stream.

Server wraps one nq_server: submit(N, queens) admits a counting request (or
returns None when the server is full), poll() returns finished (ticket, count)
pairs. run_stream() replays requests at their arrival times: each is submitted
when due (kept in a host backlog while the server is full), completions are
polled continuously, and the latency of a request is completion time minus
arrival time.
"""
from __future__ import annotations

import ctypes
import time
from collections import deque

from . import nq


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_n", ctypes.c_int32), ("request_slots", ctypes.c_int32),
                ("stack_slots", ctypes.c_int32), ("block", ctypes.c_int32),
                ("ring_records", ctypes.c_uint64), ("idle_ms", ctypes.c_uint32),
                ("reserved", ctypes.c_int32 * 3)]


def _declare():
    lib = nq.lib()
    if getattr(lib, "_serve_declared", False):
        return lib
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.nq_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]
    lib.nq_server_submit.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(nq.Queen),
                                     ctypes.c_int, u64p]
    lib.nq_server_poll.argtypes = [ctypes.c_void_p, u64p, u64p, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]
    lib.nq_server_stats.argtypes = [ctypes.c_void_p, u64p, u64p, u64p, u64p]
    lib.nq_server_destroy.argtypes = [ctypes.c_void_p]
    for f in (lib.nq_server_create, lib.nq_server_submit, lib.nq_server_poll,
              lib.nq_server_stats, lib.nq_server_destroy):
        f.restype = ctypes.c_int
    lib._serve_declared = True
    return lib


class Server:
    def __init__(self, max_n=20, request_slots=64, stack_slots=0, block=256,
                 ring_records=1 << 25, idle_ms=200):
        lib = _declare()
        cfg = ServerConfig(int(max_n), int(request_slots), int(stack_slots), int(block),
                           int(ring_records), int(idle_ms), (0, 0, 0))
        h = ctypes.c_void_p()
        nq._check(lib.nq_server_create(ctypes.byref(cfg), ctypes.byref(h)), "nq_server_create")
        self._h = h
        self._buf = 4096
        self._tk = (ctypes.c_uint64 * self._buf)()
        self._ct = (ctypes.c_uint64 * self._buf)()

    def submit(self, n: int, queens) -> int | None:
        """Ticket of the admitted request, or None if the server is full."""
        k = len(queens)
        arr = (nq.Queen * max(k, 1))(*[nq.Queen(int(r), int(c)) for r, c in queens])
        t = ctypes.c_uint64()
        rc = nq.lib().nq_server_submit(self._h, int(n), arr, k, ctypes.byref(t))
        if rc == nq.NQ_EBUSY:
            return None
        nq._check(rc, "nq_server_submit")
        return int(t.value)

    def poll(self) -> list[tuple[int, int]]:
        got = ctypes.c_int()
        nq._check(nq.lib().nq_server_poll(self._h, self._tk, self._ct, self._buf,
                                          ctypes.byref(got)), "nq_server_poll")
        return [(int(self._tk[i]), int(self._ct[i])) for i in range(got.value)]

    def stats(self) -> dict:
        v = [ctypes.c_uint64() for _ in range(4)]
        nq._check(nq.lib().nq_server_stats(self._h, *[ctypes.byref(x) for x in v]),
                  "nq_server_stats")
        return dict(zip(("submitted", "completed", "launches", "published"),
                        (int(x.value) for x in v)))

    def close(self):
        if self._h:
            rc = nq.lib().nq_server_destroy(self._h)
            self._h = None
            nq._check(rc, "nq_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_stream(server: Server, requests: list[dict], time_scale: float = 1.0,
               timeout_s: float = 600.0) -> dict:
    """Replay requests ({"t": arrival seconds, "n": N, "queens": [...]}) on server.

    Returns {"answers": {request index: count}, "latency_s": {index: seconds},
    "wall_s": ..., "busy_retries": ...}."""
    order = sorted(range(len(requests)), key=lambda i: requests[i]["t"])
    pending = deque(order)          # not yet due or waiting for admission
    backlog: deque[int] = deque()   # due but refused (server full)
    ticket_of: dict[int, int] = {}
    arrival: dict[int, float] = {}
    answers: dict[int, int] = {}
    latency: dict[int, float] = {}
    retries = 0
    t0 = time.perf_counter()
    while len(answers) < len(requests):
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError(f"{len(requests) - len(answers)} requests unanswered")
        while pending and requests[pending[0]]["t"] * time_scale <= now:
            i = pending.popleft()
            arrival[i] = t0 + requests[i]["t"] * time_scale
            backlog.append(i)
        while backlog:
            i = backlog[0]
            t = server.submit(requests[i]["n"], requests[i]["queens"])
            if t is None:
                retries += 1
                break
            backlog.popleft()
            ticket_of[t] = i
        for t, cnt in server.poll():
            i = ticket_of.pop(t)
            answers[i] = cnt
            latency[i] = time.perf_counter() - arrival[i]
        if not backlog and pending and not ticket_of:
            wait = t0 + requests[pending[0]]["t"] * time_scale - time.perf_counter()
            if wait > 0:
                time.sleep(min(wait, 0.01))
        else:
            time.sleep(20e-6)
    return {"answers": answers, "latency_s": latency, "wall_s": time.perf_counter() - t0,
            "busy_retries": retries}
