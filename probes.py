"""Command-line driver of the measurement probes (include/nq.h, "Measurement").

    python probes.py alu     # integer issue rates (the roofline)
    python probes.py smem    # shared-memory access patterns

``smem`` runs one launch per pattern, in the order of CASES, and prints one JSON
line per launch with what a conflict-free access pattern needs: for each warp
instruction, the phases with at least one active lane (128-bit accesses are
served 8 lanes per phase, 64-bit 16, 32-bit 32) and the fewest
wavefronts the active lanes' bytes could take (ceil(active bytes / 128)). Read
beside a profiler's shared-memory wavefront and bank-conflict counters for the
same launches, these tell bank conflicts (distinct words on one bank within a
phase) apart from phases that are merely sparse.
"""
from __future__ import annotations

import json
import math
import sys

from paper_2511_12009_gb300 import nq

# (kind, lane mask, density out of 32, what it is)
CASES = [
    (0, 0xFFFFFFFF, 32, "16-byte loads, interleaved frames, all lanes"),
    (0, 0x000000FF, 32, "16-byte loads, interleaved frames, lanes 0-7 (one phase)"),
    (0, 0x01010101, 32, "16-byte loads, interleaved frames, one lane in each phase"),
    (0, 0x0F0F0F0F, 32, "16-byte loads, interleaved frames, four lanes in each phase"),
    (0, 0xFFFFFFFF, 8, "16-byte loads, interleaved frames, each lane active with p = 1/4"),
    (1, 0xFFFFFFFF, 32, "16-byte stores, interleaved frames, all lanes"),
    (1, 0x01010101, 32, "16-byte stores, interleaved frames, one lane in each phase"),
    (1, 0xFFFFFFFF, 8, "16-byte stores, interleaved frames, each lane active with p = 1/4"),
    (2, 0xFFFFFFFF, 32, "4-byte loads, split arrays, all lanes"),
    (2, 0xFFFFFFFF, 8, "4-byte loads, split arrays, each lane active with p = 1/4"),
    (3, 0xFFFFFFFF, 32, "16-byte loads, per-thread contiguous stacks, all lanes"),
    (4, 0xFFFFFFFF, 32, "8-byte loads, interleaved words, all lanes"),
    (4, 0x00010001, 32, "8-byte loads, interleaved words, lanes 0 and 16"),
    (4, 0x000F000F, 32, "8-byte loads, interleaved words, lanes 0-3 and 16-19"),
    (4, 0xFFFFFFFF, 8, "8-byte loads, interleaved words, each lane active with p = 1/4"),
    (5, 0xFFFFFFFF, 8, "8-byte stores, interleaved words, each lane active with p = 1/4"),
    (6, 0xFFFFFFFF, 32, "4-byte stores, split arrays, all lanes"),
    (6, 0xFFFFFFFF, 8, "4-byte stores, split arrays, each lane active with p = 1/4"),
]
ITERS, SLOTS = 256, 8


def _binom(n: int, k: int, p: float) -> float:
    return math.comb(n, k) * p ** k * (1 - p) ** (n - k)


def expected(kind: int, mask: int, density: int) -> dict:
    """Per warp instruction: mean phases holding an active lane, and mean
    fewest wavefronts for the active bytes (both for a conflict-free pattern)."""
    width = 4 if kind in (2, 6) else 8 if kind in (4, 5) else 16
    lanes_per_phase = 128 // width
    p = min(density, 32) / 32.0
    phases, ideal = 0.0, 0.0
    for p0 in range(0, 32, lanes_per_phase):
        m = bin((mask >> p0) & ((1 << lanes_per_phase) - 1)).count("1")
        phases += 1.0 - (1.0 - p) ** m
    n = bin(mask & 0xFFFFFFFF).count("1")
    for k in range(n + 1):
        ideal += _binom(n, k, p) * math.ceil(k * width / 128)
    return {"phases_per_inst": phases, "min_wavefronts_per_inst": ideal}


def run_smem() -> list[dict]:
    out = []
    for kind, mask, density, what in CASES:
        ms = nq.probe_smem(kind, mask, density, ITERS, SLOTS)
        rec = {"kind": kind, "lane_mask": f"0x{mask:08X}", "density": density, "what": what,
               "ms": ms, "iters": ITERS, "slots": SLOTS}
        rec.update(expected(kind, mask, density))
        out.append(rec)
        print(json.dumps(rec), flush=True)
    return out


def run_alu() -> list[dict]:
    out = []
    for kind, name in enumerate(["lop3", "add", "shf", "popc", "lowbit-pick"]):
        rec = {"kind": kind, "op": name}
        rec.update(nq.probe_alu(kind))
        out.append(rec)
        print(json.dumps(rec), flush=True)
    return out


def main(argv: list[str]) -> int:
    what = argv[1] if len(argv) > 1 else "smem"
    if what == "smem":
        run_smem()
    elif what == "alu":
        run_alu()
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
