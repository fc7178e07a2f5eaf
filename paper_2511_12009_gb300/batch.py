"""Batched counting (binding of the nq_batch_* calls): the prefix sets of several
board sizes searched by one persistent kernel launch replayed from a CUDA graph,
next to the same work as one plain launch per board."""
from __future__ import annotations

import ctypes

import numpy as np

from . import nq


class Batch:
    def __init__(self, ns, ds=None, config: nq.Config | None = None):
        self.ns = [int(n) for n in ns]
        k = len(self.ns)
        arr_n = (ctypes.c_int * k)(*self.ns)
        arr_d = (ctypes.c_int * k)(*[int(d) for d in ds]) if ds is not None else None
        handle = ctypes.c_void_p()
        cfg = ctypes.byref(config) if config is not None else None
        nq._check(nq.lib().nq_batch_create(arr_n, arr_d, k, cfg, ctypes.byref(handle)),
                  "nq_batch_create")
        self._h = handle

    def info(self) -> dict:
        rec = ctypes.c_uint64()
        md, mn, g, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nq._check(nq.lib().nq_batch_info(self._h, ctypes.byref(rec), ctypes.byref(md),
                                         ctypes.byref(mn), ctypes.byref(g), ctypes.byref(b)),
                  "nq_batch_info")
        return {"records": rec.value, "min_d": md.value, "max_n": mn.value, "grid": g.value,
                "block": b.value}

    def _run(self, fn, stream) -> tuple[list[int], float]:
        k = len(self.ns)
        out = (ctypes.c_uint64 * k)()
        ms = ctypes.c_float()
        nq._check(fn(self._h, nq._stream_handle(stream), out, ctypes.byref(ms)), fn.__name__)
        return [int(v) for v in out], float(ms.value)

    def run(self, stream=None):
        """One graph replay: (totals per board in the given order, milliseconds)."""
        return self._run(nq.lib().nq_batch_run, stream)

    def run_separate(self, stream=None):
        """One plain launch per board, back to back: (totals, milliseconds)."""
        return self._run(nq.lib().nq_batch_run_separate, stream)

    def counts(self, board: int) -> np.ndarray:
        num = ctypes.c_uint64()
        nq._check(nq.lib().nq_batch_counts(self._h, board, None, 0, ctypes.byref(num)),
                  "nq_batch_counts")
        out = np.zeros(max(num.value, 1), dtype=np.uint64)
        nq._check(nq.lib().nq_batch_counts(self._h, board, out.ctypes.data, num.value,
                                           ctypes.byref(num)), "nq_batch_counts")
        return out[:num.value]

    def close(self):
        if self._h:
            nq.lib().nq_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
