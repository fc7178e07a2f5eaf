"""CPU tests of two host-side pieces of the C ABI: the static multi-worker split
(Section 4.5) pinned to the paper's 27-Queens run log, and a shared-memory bank
simulator over the stack addresses the search kernel uses (Section 3.1)."""
import json
import os

import numpy as np
import pytest

from paper_2511_12009_gb300 import nq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- static split (Section 4.5) -----------------------------------------------

def test_ratio_split_reproduces_the_27_queens_log():
    g = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    total = g["n27_subproblems"]["value"]
    part = nq.partition(total, 8, g["n27_partition"]["ratios"])
    assert [c for _, c in part] == g["n27_partition"]["per_gpu"]
    # contiguous slices covering the list once, in order
    assert part[0][0] == 0
    for (f0, c0), (f1, _) in zip(part, part[1:]):
        assert f1 == f0 + c0
    assert part[-1][0] + part[-1][1] == total


def test_ratio_split_is_single_precision():
    """Double-precision products miss the log's counts: the rule is float32."""
    g = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    total = g["n27_subproblems"]["value"]
    ratios = g["n27_partition"]["ratios"]
    f64 = [int(r * total) for r in ratios[:7]]
    assert f64 != g["n27_partition"]["per_gpu"][:7]


@pytest.mark.parametrize("n,k", [(0, 1), (0, 3), (1, 1), (7, 8), (10, 3), (1000003, 7), (2**40 + 5, 64)])
def test_uniform_split(n, k):
    part = nq.partition(n, k)
    assert [c for _, c in part[:-1]] == [n // k] * (k - 1)
    assert part[-1][1] == n - (k - 1) * (n // k)
    assert sum(c for _, c in part) == n


def test_split_rejects_bad_arguments():
    with pytest.raises(nq.NQError):
        nq.partition(10, 0)
    with pytest.raises(nq.NQError):
        nq.partition(10, 2, [1.5, 0.0])
    with pytest.raises(nq.NQError):
        nq.partition(10, 2, [float("nan"), 0.5])
    with pytest.raises(nq.NQError):
        nq.partition(10, 3, [0.7, 0.7, 0.0])  # shares beyond n


# --- bank simulator (Section 3.1) -----------------------------------------------

BANKS, BANK_BYTES, PHASE_BYTES = 32, 4, 128


def phase_degrees(addrs, width):
    """Accesses of one warp instruction (addrs[lane] or None for an inactive lane,
    `width` bytes each) served in phases of 128 / width lanes; within a phase, the
    words of one bank that differ are served one after another. Returns the
    largest number of distinct words on one bank, per phase."""
    per_phase = PHASE_BYTES // width
    out = []
    for p0 in range(0, 32, per_phase):
        words_by_bank = {}
        for a in addrs[p0:p0 + per_phase]:
            if a is None:
                continue
            for w in range(a // BANK_BYTES, (a + width) // BANK_BYTES):
                words_by_bank.setdefault(w % BANKS, set()).add(w)
        out.append(max((len(v) for v in words_by_bank.values()), default=0))
    return out


def test_simulator_catches_a_conflicting_layout():
    # per-thread contiguous stacks of 8 frames: lanes of a phase sit 128 bytes apart
    addrs = [(t * 8 + 3) * 16 for t in range(32)]
    assert max(phase_degrees(addrs, 16)) == 8
    # 32-bit words at a 16-byte lane stride: 4-way
    assert max(phase_degrees([t * 16 for t in range(32)], 4)) == 4


# Accesses each layout's step makes: (field, width) -- 16-byte frames move whole;
# WT and WTM also write the avail word alone; WT32 moves single words.
ACCESSES = {
    "paper": [(0, 16)], "reg": [(0, 16)], "regm": [(0, 16)],
    "wt": [(0, 16), (3, 4)], "wtm": [(0, 16), (3, 4)],
    "wt32": [(0, 4), (1, 4), (2, 4), (3, 4)], "wt32a": [(0, 4), (1, 4), (2, 4), (3, 4)],
    "regp": [(0, 16)],
    "regz": [(0, 4), (1, 4), (2, 4), (3, 4)], "regpz": [(0, 4), (1, 4), (2, 4), (3, 4)],
    "avail": [(3, 4)],
}
SPLIT_WORDS = {"regz", "regpz"}  # built for 256-thread blocks only
KNOWN_4WAY = {("wt", 3), ("wtm", 3)}  # the lone avail-word stores of WT and WTM


@pytest.mark.parametrize("layout", sorted(ACCESSES))
@pytest.mark.parametrize("block", [64, 128, 160, 192, 256, 512])
def test_stack_layouts_bank_conflicts(layout, block):
    if layout in SPLIT_WORDS and block != 256:
        pytest.skip("split-word frames are compiled for 256-thread blocks")
    rng = np.random.default_rng(block)
    slots = 12
    for trial in range(40):
        depth = rng.integers(0, slots, size=32)
        active = rng.random(32) < (1.0 if trial % 4 == 0 else 0.4)
        warp = int(rng.integers(0, block // 32))
        for field, width in ACCESSES[layout]:
            addrs = [nq.stack_offset(layout, block, slots, warp * 32 + t, int(depth[t]), field)
                     if active[t] else None for t in range(32)]
            deg = max(phase_degrees(addrs, width))
            if (layout, field) in KNOWN_4WAY and width == 4:
                # the lone 32-bit avail store into 16-byte frames: lanes t, t+8,
                # t+16, t+24 share a bank (why REGM / REG store whole frames)
                assert deg <= 4
            else:
                assert deg <= 1, (layout, block, field, depth.tolist())


def test_wt_avail_store_is_four_way_with_every_lane():
    addrs = [nq.stack_offset("wt", 256, 12, t, 5, 3) for t in range(32)]
    assert max(phase_degrees(addrs, 4)) == 4


def test_stack_offset_rejects_bad_arguments():
    for args in [(99, 256, 8, 0, 0, 0), ("regm", 100, 8, 0, 0, 0), ("regm", 256, 8, 256, 0, 0),
                 ("regm", 256, 8, 0, 8, 0), ("regm", 256, 8, 0, 0, 4)]:
        with pytest.raises(nq.NQError):
            nq.stack_offset(*args)


@pytest.mark.parametrize("layout", sorted(SPLIT_WORDS))
def test_split_words_one_bank_per_lane(layout):
    """Split-word frames: every word of thread t sits in bank t mod 32, at any
    slot and field, so a warp's 32-bit accesses -- by any subset of lanes, at any
    mix of depths -- touch distinct banks (one wavefront, nothing to conflict)."""
    for t in range(256):
        for slot in (0, 1, 5, 11):
            for field in range(4):
                off = nq.stack_offset(layout, 256, 12, t, slot, field)
                assert off % 4 == 0 and (off // 4) % 32 == t % 32
    # distinct words for distinct (thread, slot, field)
    offs = {nq.stack_offset(layout, 256, 12, t, k, f)
            for t in range(256) for k in range(12) for f in range(4)}
    assert len(offs) == 256 * 12 * 4 and max(offs) < 256 * 12 * 16
    with pytest.raises(nq.NQError):
        nq.stack_offset(layout, 128, 12, 0, 0, 0)
