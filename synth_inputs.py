"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds random-number generation only: it computes nothing of the
counting method. Both the CUDA path and the CPU oracle receive what it draws as
plain inputs (ranks, child choices, constraint cells, arrival times), so the two
sides never share arithmetic.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser with the
golden-ratio increment), written out here from that published definition.
"""
from __future__ import annotations

import math

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream: state += 0x9E3779B97F4A7C15, then a 3-step xor-shift-multiply mix."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("n must be positive")
        limit = (1 << 64) - ((1 << 64) % n)
        while True:
            v = self.next_u64()
            if v < limit:
                return v % n

    def uniform(self) -> float:
        """Uniform float in (0, 1]: 53 random bits."""
        return ((self.next_u64() >> 11) + 1) / float(1 << 53)


def sample_ranks(seed: int, total: int, k: int) -> list[int]:
    """k distinct ranks drawn uniformly from [0, total), in draw order."""
    if k > total:
        raise ValueError("cannot draw more distinct ranks than exist")
    g = SplitMix64(seed)
    seen: set[int] = set()
    out: list[int] = []
    while len(out) < k:
        r = g.below(total)
        if r not in seen:
            seen.add(r)
            out.append(r)
    return out


def raw_u64(seed: int, count: int) -> list[int]:
    """count raw 64-bit draws (used as child choices of a seeded random walk)."""
    g = SplitMix64(seed)
    return [g.next_u64() for _ in range(count)]


def _attacks(a: tuple[int, int], b: tuple[int, int]) -> bool:
    """Chess rule: same row, same column or same diagonal."""
    return a[0] == b[0] or a[1] == b[1] or abs(a[0] - b[0]) == abs(a[1] - b[1])


def constraint_set(g: SplitMix64, n: int, k: int) -> list[tuple[int, int]]:
    """k queens on distinct cells of an n x n board, no two attacking each other,
    drawn uniformly over cells by rejection of whole sets."""
    while True:
        qs: list[tuple[int, int]] = []
        ok = True
        for _ in range(k):
            cell = (g.below(n), g.below(n))
            if any(_attacks(cell, q) for q in qs):
                ok = False
                break
            qs.append(cell)
        if ok:
            return qs


def request_stream(seed: int, count: int, n_lo: int, n_hi: int, k_lo: int, k_hi: int,
                   rate_per_s: float) -> list[dict]:
    """Seeded Poisson request stream: exponential inter-arrival times at rate_per_s,
    board size N uniform in [n_lo, n_hi], k uniform in [k_lo, k_hi] non-attacking
    constraint queens. Each request: {"t": arrival seconds, "n": N, "queens": [...]}."""
    g = SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(g.uniform()) / rate_per_s if rate_per_s > 0 else 0.0
        n = n_lo + g.below(n_hi - n_lo + 1)
        k = k_lo + g.below(k_hi - k_lo + 1)
        out.append({"id": i, "t": t, "n": n, "queens": constraint_set(g, n, k)})
    return out


def sample_indices(seed: int, population: int, k: int) -> list[int]:
    """k distinct indices in [0, population), sorted (for sampled parity checks)."""
    k = min(k, population)
    return sorted(sample_ranks(seed, population, k)) if k else []
