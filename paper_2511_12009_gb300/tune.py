"""Autotuner for the search launch.

Axes: prefix depth d, stack layout, threads per block, claim order, and the
work chunk (subproblems a lane claims per atomic). Each candidate is timed by
the kernel's own CUDA events inside nq_total_ex (best of `reps`); every
candidate must return the same total. The search is staged (depth, then
layout, then block and order, then chunk), each stage keeping the best of the
previous ones, so a board size costs a few dozen launches. Results are cached
in a JSON file keyed by device name, SM count, a hash of libnq's sources (a
kernel change invalidates every entry) and board size (``NQ_TUNE_CACHE``,
default ``paper_2511_12009_gb300/_build/tune_cache.json``).
"""
from __future__ import annotations

import json
import os
import threading

from . import nq

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.environ.get("NQ_TUNE_CACHE", os.path.join(_HERE, "_build", "tune_cache.json"))
_lock = threading.Lock()
FIELDS = ("layout", "block", "blocks_per_sm", "order", "d", "claim")


def _source_hash() -> str:
    """sha256 (first 16 hex digits) over libnq's sources and headers."""
    import hashlib
    from . import _build
    h = hashlib.sha256()
    for path in sorted(_build._inputs()):
        h.update(os.path.basename(path).encode())
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}|{_source_hash()}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, rec: dict):
    with _lock:
        data = _load()
        data[key] = rec
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)


def measure(n: int, cfg: dict, reps: int = 2) -> tuple[float, int]:
    """Best kernel milliseconds of nq_total_ex over `reps` runs, and the total."""
    best, total = None, None
    c = nq.make_config(**cfg)
    for _ in range(reps):
        r = nq.total_ex(n, c)
        if total is not None and r["total"] != total:
            raise RuntimeError(f"N={n}: totals differ between runs of {cfg}")
        total = r["total"]
        best = r["kernel_ms"] if best is None else min(best, r["kernel_ms"])
    return best, total


def _depths(n: int, max_records: int) -> list[int]:
    d0 = nq.default_depth(n)
    out = []
    for d in (d0 - 1, d0, d0 + 1):
        if 1 <= d <= max(1, n - 2) and nq.prefix_count(n, d) <= max_records:
            out.append(d)
    return out or [d0]


def tune(n: int, reps: int = 2, max_records: int = 64_000_000,
         layouts=("regp", "regm", "reg", "wt"), blocks=(128, 192, 256, 512), claims=(1, 2, 4),
         verbose=False) -> dict:
    """Tune the launch for board size n; returns the best config (also cached)."""
    key = f"{_device_key()}|N={n}"
    tried = []

    def run(cfg):
        ms, total = measure(n, cfg, reps)
        tried.append({**cfg, "ms": ms})
        if verbose:
            print(f"  N={n} {cfg} -> {ms:.3f} ms", flush=True)
        return ms, total

    best = {"layout": 0, "block": 0, "blocks_per_sm": 0, "order": 0, "d": nq.default_depth(n),
            "claim": 0}
    best_ms, ref_total = run(best)

    def stage(variants):
        nonlocal best, best_ms
        for change in variants:
            cfg = {**best, **change}
            if cfg == best:
                continue
            ms, total = run(cfg)
            if total != ref_total:
                raise RuntimeError(f"N={n}: {cfg} gives {total}, expected {ref_total}")
            if ms < best_ms:
                best, best_ms = cfg, ms

    stage([{"d": d} for d in _depths(n, max_records)])
    stage([{"layout": nq.LAYOUTS[lay]} for lay in layouts])
    stage([{"block": b, "order": o} for b in blocks for o in (0, 1)])
    stage([{"claim": c} for c in claims])
    rec = {"config": best, "ms": best_ms, "total": ref_total, "tried": tried}
    _store(key, rec)
    return best


def cached(n: int) -> dict | None:
    rec = _load().get(f"{_device_key()}|N={n}")
    return rec["config"] if rec else None


def best_config(n: int) -> nq.Config:
    """The cached tuned config for board size n, else the library defaults."""
    cfg = cached(n)
    return nq.make_config(**cfg) if cfg else nq.make_config(d=nq.default_depth(n))


def tune_batch(ns, reps: int = 1, layouts=("regp", "regm", "reg"), blocks=(192, 256),
               claims=(2, 4), depth_offsets=(-1, 1), verbose=False) -> dict:
    """Tune a batched launch over boards ns, staged like tune(): the prefix
    depths (every board's tuned or default depth, shifted together by each of
    depth_offsets), then the stack layout, then the block size (0 = the one
    keeping the most threads resident) and claim order, then the claim chunk --
    each stage keeping the best so far. Every candidate is one captured graph
    timed by its own replays (best of `reps`) and must give the same totals.
    Returns {"ds": [...], "config": {...}, "ms": ..., "tried": [...]} (cached)."""
    from .batch import Batch
    base_ds = []
    for n in ns:
        c = cached(n)
        base_ds.append(c["d"] if c else nq.default_depth(n))
    tried = []
    ref = None

    def run(ds, cfg):
        nonlocal ref
        with Batch(ns, ds, nq.make_config(**cfg)) as b:
            ms = None
            for _ in range(reps):
                tot, t = b.run()
                if ref is not None and tot != ref:
                    raise RuntimeError(f"batch totals differ for {ds} {cfg}")
                ref = tot
                ms = t if ms is None else min(ms, t)
        tried.append({"ds": list(ds), **cfg, "ms": ms})
        if verbose:
            print(f"  batch ds={ds} {cfg} -> {ms:.3f} ms", flush=True)
        return ms

    best_ds = list(base_ds)
    best = {"layout": 0, "block": 0, "blocks_per_sm": 0, "order": 0, "d": 0, "claim": 0}
    best_ms = run(best_ds, best)
    for off in depth_offsets:
        ds = [min(max(1, d + off), max(1, n - 2)) for d, n in zip(base_ds, ns)]
        if ds != best_ds:
            ms = run(ds, best)
            if ms < best_ms:
                best_ds, best_ms = ds, ms

    def stage(variants):
        nonlocal best, best_ms
        for change in variants:
            cfg = {**best, **change}
            if cfg == best:
                continue
            ms = run(best_ds, cfg)
            if ms < best_ms:
                best, best_ms = cfg, ms

    stage([{"layout": nq.LAYOUTS[lay]} for lay in layouts])
    stage([{"block": b, "order": o} for b in (0,) + tuple(blocks) for o in (0, 1)])
    stage([{"claim": c} for c in claims])
    rec = {"ds": best_ds, "config": best, "ms": best_ms, "totals": ref, "tried": tried}
    _store(f"{_device_key()}|batch={','.join(map(str, ns))}", rec)
    return rec


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="tune the search launch per board size")
    ap.add_argument("n", type=int, nargs="+")
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()
    for n in a.n:
        print(n, tune(n, reps=a.reps, verbose=True))
