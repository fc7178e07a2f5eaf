"""Counting one board across several workers, one process per GPU (Section 4.5).

The subproblems of a board (its depth-d prefix set in canonical order) are
independent: workers share no data while they search, and the one exchange is
the sum of their totals at the end (a single 64-bit all-reduce). Two splits:

- ``static``: nq_partition's contiguous slices, uniform or by ratios (the
  paper's multi-GPU scheme, Section 4.5), each slice counted in pieces of at
  most ``chunk`` subproblems;
- ``lease`` (not in the paper): workers take chunks of consecutive
  subproblems from one shared counter (a torch.distributed Store ``add``), so
  a worker whose subtrees turn out light simply takes more chunks; nothing
  waits on another worker until the final sum.

Checkpoint / resume (not in the paper; its 27-Queens run took 28 days): with
``checkpoint=path`` every worker appends, per counted piece, a record (first
subproblem index, the piece's per-subproblem counts, a CRC-32) to its own log
``path.rank<r>``. A restarted job -- with any number of workers, either split,
any chunk size -- first reads every worker's log, keeps each complete record
whose CRC checks (a record cut short by a crash is dropped with everything
after it in that log), and counts only the subproblems not yet covered. The
log header names the board, depth and number of subproblems; a log of another
job is refused, and so are two records that give one subproblem different
counts.

Counting itself goes through ``counter(records) -> counts``; the default runs
libnq's search kernel on this process's GPU.
"""
from __future__ import annotations

import bisect
import glob
import json
import os
import struct
import zlib
from typing import Callable

import numpy as np

from . import nq

MAGIC = b"NQCK1\n"
_REC = struct.Struct("<QQI")  # first subproblem, number of counts, crc32 of the counts


class CheckpointError(RuntimeError):
    pass


def gpu_counter(device=None, config: nq.Config | None = None,
                split: bool = False) -> Callable[[np.ndarray], np.ndarray]:
    """Per-prefix solution counts of host records, on this process's GPU.
    split: count through nq_count_split (each record expanded a few rows on the
    host so that a piece of few heavy subtrees still fills the GPU)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)

    def count(records: np.ndarray) -> np.ndarray:
        if len(records) == 0:
            return np.zeros(0, dtype=np.uint64)
        if split:
            with torch.cuda.device(dev):
                return np.asarray(nq.count_split(records, -1, config)["counts"],
                                  dtype=np.uint64).copy()
        d_pre = nq.to_device(records, dev)
        counts = torch.zeros(len(records), dtype=torch.int64, device=dev)
        meta = records["meta"]
        min_d = int(((meta >> 7) & 31).min())
        max_n = int(((meta >> 2) & 31).max())
        with torch.cuda.device(dev):
            stream = torch.cuda.current_stream(dev)
            nq.count_ex(d_pre, min_d, max_n, counts, None, None, config, stream)
            nq.sync(stream)
        return counts.cpu().numpy().view(np.uint64).copy()

    return count


def _weighted(records: np.ndarray, counts: np.ndarray) -> int:
    w = (records["meta"] & 3).astype(np.uint64)
    return int((w * np.asarray(counts, dtype=np.uint64)).sum(dtype=np.uint64))


class _Log:
    """One worker's append-only checkpoint log."""

    def __init__(self, path: str, header: dict):
        fresh = not os.path.exists(path) or os.path.getsize(path) == 0
        self.f = open(path, "ab")
        if fresh:
            self.f.write(MAGIC + json.dumps(header, sort_keys=True).encode() + b"\n")
            self._sync()

    def _sync(self):
        self.f.flush()
        os.fsync(self.f.fileno())

    def append(self, first: int, counts: np.ndarray):
        data = np.ascontiguousarray(counts, dtype=np.uint64).tobytes()
        self.f.write(_REC.pack(first, len(counts), zlib.crc32(data)) + data)
        self._sync()

    def close(self):
        self.f.close()


class Done:
    """Subproblem ranges already counted: sorted, disjoint [lo, hi) with counts."""

    def __init__(self):
        self.lo: list[int] = []
        self.hi: list[int] = []
        self.counts: list[np.ndarray] = []

    def add(self, lo: int, counts: np.ndarray, where: str = ""):
        hi = lo + len(counts)
        if hi == lo:
            return
        # every range it overlaps must agree on the shared subproblems
        k = max(0, bisect.bisect_right(self.lo, lo) - 1)
        while k < len(self.lo) and self.lo[k] < hi:
            if lo < self.hi[k]:
                a, b = max(lo, self.lo[k]), min(hi, self.hi[k])
                if not np.array_equal(counts[a - lo:b - lo],
                                      self.counts[k][a - self.lo[k]:b - self.lo[k]]):
                    raise CheckpointError(f"{where}: subproblems {a}..{b - 1} recorded with two counts")
            k += 1
        # keep only the parts not yet covered
        for a, b in self.missing(lo, hi):
            k = bisect.bisect_right(self.lo, a)
            self.lo.insert(k, a)
            self.hi.insert(k, b)
            self.counts.insert(k, np.asarray(counts[a - lo:b - lo], dtype=np.uint64).copy())

    def missing(self, lo: int, hi: int) -> list[tuple[int, int]]:
        """Sub-ranges of [lo, hi) not covered."""
        out, pos = [], lo
        k = max(0, bisect.bisect_right(self.lo, lo) - 1)
        while pos < hi and k < len(self.lo):
            if self.hi[k] <= pos:
                k += 1
                continue
            if self.lo[k] >= hi:
                break
            if self.lo[k] > pos:
                out.append((pos, self.lo[k]))
            pos = max(pos, self.hi[k])
            k += 1
        if pos < hi:
            out.append((pos, hi))
        return out

    def covered(self) -> int:
        return sum(b - a for a, b in zip(self.lo, self.hi))

    def items(self):
        return zip(self.lo, self.counts)


def read_checkpoint(path: str, header: dict) -> Done:
    """Every worker's log of `path`, merged. Raises CheckpointError for a log
    written for another job or two records that disagree."""
    done = Done()
    for fn in sorted(glob.glob(glob.escape(path) + ".rank*")):
        with open(fn, "rb") as f:
            blob = f.read()
        if not blob:
            continue
        if not blob.startswith(MAGIC):
            raise CheckpointError(f"{fn}: not a checkpoint log")
        end = blob.find(b"\n", len(MAGIC))
        if end < 0:
            raise CheckpointError(f"{fn}: header cut short")
        try:
            got = json.loads(blob[len(MAGIC):end])
        except ValueError as e:
            raise CheckpointError(f"{fn}: unreadable header") from e
        if got != header:
            raise CheckpointError(f"{fn}: written for {got}, not {header}")
        pos = end + 1
        while pos + _REC.size <= len(blob):
            first, k, crc = _REC.unpack_from(blob, pos)
            body = blob[pos + _REC.size: pos + _REC.size + 8 * k]
            if len(body) != 8 * k or zlib.crc32(body) != crc or first + k > header["records"]:
                break  # cut short by a crash, or damaged: the rest of this log is dropped
            done.add(int(first), np.frombuffer(body, dtype=np.uint64), fn)
            pos += _REC.size + 8 * k
    return done


def records_digest(records: np.ndarray) -> str:
    """sha256 (first 16 hex digits) of a record array: names a sample in a log."""
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(records, dtype=nq.PREFIX_DTYPE).tobytes()
                          ).hexdigest()[:16]


def count_board(n: int, d: int | None = None, *, rank: int = 0, world: int = 1,
                mode: str = "lease", ratios=None, chunk: int = 1 << 16, store=None,
                job: str = "nq", counter: Callable | None = None, checkpoint: str | None = None,
                on_piece: Callable[[int, int], None] | None = None,
                records: np.ndarray | None = None) -> dict:
    """Count the N-Queens solutions of an n x n board with `world` workers, this
    process being worker `rank`.

    records: count these subproblems (records of board n) instead of the
    board's whole depth-d prefix set -- a sample of a board too large to count
    whole (the paper's 27-Queens run, Section 4.5); d is then the records'
    smallest depth, "total" their weighted sum, and the checkpoint header also
    carries the records' digest, so that a log of another sample is refused.

    mode "static": worker `rank` counts its nq_partition slice (ratios as
    there, None = uniform) in pieces of at most `chunk` subproblems. mode
    "lease": chunk i = subproblems [i * chunk, (i + 1) * chunk) goes to the
    worker whose store.add(job + "/cursor", 1) returned i + 1 (`store` is
    required when world > 1; a single worker counts locally).
    `on_piece(lo, hi)` runs after each piece is counted and logged: a worker
    that fails there leaves nothing half-recorded.

    With a torch.distributed process group of `world` ranks up, "total" is the
    sum over all workers (one all-reduce); otherwise it is this worker's part.
    Returns {"total", "local_total", "pieces": {lo: counts} counted here,
    "resumed": subproblems taken from the checkpoint, "records"}.
    """
    import torch.distributed as dist
    if d is None:
        d = nq.default_depth(n)
    if mode not in ("static", "lease"):
        raise ValueError("mode is 'static' or 'lease'")
    if chunk < 1:
        raise ValueError("chunk >= 1")
    if world > 1 and mode == "lease" and store is None:
        raise ValueError("leasing across workers needs a shared store")
    if counter is None:
        counter = gpu_counter()
    if records is None:
        records = nq.enumerate_prefixes(n, d)
        m = len(records)
        header = {"n": int(n), "d": int(d), "records": int(m)}
    else:
        records = np.ascontiguousarray(records, dtype=nq.PREFIX_DTYPE)
        m = len(records)
        if m and int(((records["meta"] >> 2) & 31).max()) != n:
            raise ValueError("records of another board size")
        d = int(((records["meta"] >> 7) & 31).min()) if m else 0
        header = {"n": int(n), "d": int(d), "records": int(m), "sample": records_digest(records)}

    done = read_checkpoint(checkpoint, header) if checkpoint is not None else Done()
    group = dist.is_available() and dist.is_initialized() and world > 1
    if group and (dist.get_world_size() != world or dist.get_rank() != rank):
        raise ValueError(f"worker {rank} of {world}, but the process group has rank "
                         f"{dist.get_rank()} of {dist.get_world_size()}")
    if not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    if group:
        dist.barrier()  # every worker has read the logs before anyone appends
    log = _Log(f"{checkpoint}.rank{rank}", header) if checkpoint is not None else None

    def units():
        if mode == "static":
            first, cnt = nq.partition(m, world, ratios)[rank]
            for lo in range(first, first + cnt, chunk):
                yield lo, min(first + cnt, lo + chunk)
        else:
            n_chunks = (m + chunk - 1) // chunk
            local = 0
            while True:
                if store is not None:
                    i = int(store.add(f"{job}/cursor", 1)) - 1
                else:
                    i, local = local, local + 1
                if i >= n_chunks:
                    return
                yield i * chunk, min(m, (i + 1) * chunk)

    local_total = 0
    pieces: dict[int, np.ndarray] = {}
    try:
        for lo0, hi0 in units():
            for lo, hi in done.missing(lo0, hi0):
                counts = np.asarray(counter(records[lo:hi]), dtype=np.uint64)
                if len(counts) != hi - lo:
                    raise RuntimeError("counter returned the wrong number of counts")
                local_total += _weighted(records[lo:hi], counts)
                pieces[lo] = counts
                if log is not None:
                    log.append(lo, counts)
                if on_piece is not None:
                    on_piece(lo, hi)
    finally:
        if log is not None:
            log.close()

    # the checkpoint's part is added once, by worker 0
    resumed_total = 0
    if rank == 0:
        for lo, c in done.items():
            resumed_total += _weighted(records[lo:lo + len(c)], c)
    total = local_total + resumed_total
    if group:
        import torch
        t = torch.tensor([total], dtype=torch.int64)
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t)
        total = int(t.item())
    return {"total": total, "local_total": local_total + resumed_total, "pieces": pieces,
            "resumed": done.covered(), "records": m}
