"""A step-by-step model of one lane of the default search kernel (layout REGM),
and of its form with the last row pushed (REGP), checked on the CPU against
the oracle: the multiply-add form of the step (Algorithm 2 with Algorithm 3's
last-row rule, or without it and a solution recognised by a full column mask),
the predicated push / save / pop tail, the two sentinel frames and the 31-step
rounds between bookkeeping points. It pins the arithmetic and stack bounds the kernel relies on -- the
exact sums behind the multiply-adds, N - d stack slots per lane, and an idle
lane never popping below its stack within a round -- on whole prefix sets,
not the kernel's code itself (the GPU parity tests do that)."""
import pytest

from paper_2511_12009_gb300 import nq

M = 0xFFFFFFFF
STEPS_PER_ROUND = 31
# the kernel's sentinel frame for the multiply-add layouts
SENTINEL = (0xAAAAAAAA, 0xAAAAAAAA, 0xAAAAAAAA, 0x55555555)


def popc(x):
    return bin(x).count("1")


def step(state, stack, top, pushlast=False):
    """One REGM step (REGP with pushlast): returns (state, top, counted
    solution). `stack` maps slot index -> saved frame; `top` is the next free
    slot."""
    c, l, r, av = state
    p = av & ((av * M) & M)                      # av & -av
    ar = (p * M + av) & M                        # av - p
    c2 = (p + c) & M                             # cols | p
    l2 = (l * 2 + p * 2) & M                     # (ld | p) << 1
    r2 = ((((p + r) & M) * 0x80000000) >> 32)    # (rd | p) >> 1, as umulhi
    a2 = ~(c2 | l2 | r2) & M                     # free columns of the next row
    if pushlast:
        pcnt = c2 == M                           # every column holds a queen
        ppush = a2 != 0
    else:
        plast = popc(c2) == 31
        pcnt = a2 != 0 and plast
        ppush = a2 != 0 and not plast
    psave = ar != 0 and ppush
    ppop = ar == 0 and not ppush
    if psave:
        stack[top] = (c, l, r, ar)
        top += 1
    if ppop:
        top -= 1
        assert top >= 0, "popped below the stack"
        c, l, r, av = stack[top]
    elif ppush:
        c, l, r, av = c2, l2, r2, a2
    else:
        av = ar
    return (c, l, r, av), top, 1 if pcnt else 0


def search(rec, slots, pushlast=False):
    """Solutions and nodes below one record, the lane running whole rounds;
    also the deepest slot used."""
    n = (int(rec["meta"]) >> 2) & 31
    d = (int(rec["meta"]) >> 7) & 31
    last = (1 << n) - 1
    c0 = int(rec["cols"]) | (~last & M)
    l0, r0 = int(rec["ld"]), int(rec["rd"]) & last
    a0 = ~(c0 | l0 | r0) & M
    if d == n:
        return 1, 0, 0
    if d + 1 == n or a0 == 0:
        s = popc(a0)
        return s, s, 0
    stack = {0: SENTINEL, 1: SENTINEL}
    state, top = (c0, l0, r0, a0), 2
    sol = steps = 0
    deepest = top
    while True:
        for _ in range(STEPS_PER_ROUND):
            if top > 1:        # on the subproblem (top <= 1: idle on a sentinel)
                steps += 1
            state, top, s = step(state, stack, top, pushlast)
            sol += s
            deepest = max(deepest, top)
            assert top <= slots, "a frame was saved beyond the lane's last slot"
        if top <= 1:           # idle at the bookkeeping point: subproblem done
            # REGP's solutions are steps of their own
            return sol, steps if pushlast else steps + sol, deepest


@pytest.mark.parametrize("n,d", [(6, 2), (8, 3), (9, 4), (10, 3), (10, 6), (11, 5), (7, 7),
                                 (9, 8)])
def test_model_equals_oracle(orc, n, d):
    pre = nq.enumerate_prefixes(n, d)
    cols, _ = orc.prefixes(n, d)
    want, want_nodes = orc.count_prefixes(n, cols)
    slots = max(n - 1 - d, 1) + 1   # the kernel's stack for REGM
    for i, rec in enumerate(pre):
        sol, nodes, deepest = search(rec, slots)
        assert (sol, nodes) == (int(want[i]), int(want_nodes[i])), (n, d, i)
        assert deepest <= slots      # every saved frame lies in slots 2 .. slots-1


def test_idle_lane_lasts_a_round_and_no_more():
    """From the reset idle state (sentinel in registers, top at slot 1) a lane
    takes 31 steps without leaving its stack; a 32nd would pop below slot 0."""
    stack = {0: SENTINEL, 1: SENTINEL}
    state, top = SENTINEL, 1
    for _ in range(STEPS_PER_ROUND):
        state, top, s = step(state, stack, top)
        assert s == 0 and 0 <= top <= 1
    with pytest.raises(AssertionError, match="below"):
        step(state, stack, top)


def test_sentinel_never_pushes_or_counts():
    state, top, stack = SENTINEL, 1, {0: SENTINEL, 1: SENTINEL}
    for _ in range(16):
        state, top2, s = step(state, stack, top)
        assert s == 0 and top2 <= top
        top = top2


def test_slots_bound_is_tight_somewhere(orc):
    """Some N=10, d=3 subproblem uses every one of the N - d slots, so one slot
    fewer would overflow."""
    n, d = 10, 3
    slots = (n - 1 - d) + 1
    assert max(search(rec, slots)[2] for rec in nq.enumerate_prefixes(n, d)) == slots


@pytest.mark.parametrize("n,d", [(6, 2), (8, 3), (9, 4), (10, 3), (10, 6), (11, 5), (7, 7),
                                 (9, 8), (13, 4)])
def test_pushed_last_row_model_equals_oracle(orc, n, d):
    """REGP: the same counts and nodes, with N + 1 - d slots (the row N-2 frame
    may be saved), a bound some N=13, d=4 subproblem reaches."""
    pre = nq.enumerate_prefixes(n, d)
    cols, _ = orc.prefixes(n, d)
    want, want_nodes = orc.count_prefixes(n, cols)
    slots = max(n - d, 1) + 1
    deepest = 0
    for i, rec in enumerate(pre):
        sol, nodes, dp = search(rec, slots, pushlast=True)
        assert (sol, nodes) == (int(want[i]), int(want_nodes[i])), (n, d, i)
        deepest = max(deepest, dp)
    if (n, d) == (13, 4):
        assert deepest == slots


def test_pushed_last_row_sentinel_lasts_a_round():
    stack = {0: SENTINEL, 1: SENTINEL}
    state, top = SENTINEL, 1
    for _ in range(STEPS_PER_ROUND):
        state, top, s = step(state, stack, top, pushlast=True)
        assert s == 0 and 0 <= top <= 1


# --- the constrained multiply-add step (server kernel, nq_count_constrained) ----

ROW_SHIFT, ROW_INC = 27, 1 << 27
SENTINEL_C = (30 << ROW_SHIFT, 0, 0, ROW_INC - 1)   # row 30, no column, 27 candidates


def step_constrained(state, stack, top, allowed, thr):
    """One constrained step: the row rides in bits 27..31 of cols; the child's
    row takes only allowed[row + 1]; the last row is reached when the child's
    row field is >= thr = (N - 1) << 27."""
    c, l, r, av = state
    al = allowed[(c >> ROW_SHIFT) + 1]
    p = av & ((av * M) & M)
    ar = (p * M + av) & M
    c2 = (p + c + ROW_INC) & M
    l2 = (l * 2 + p * 2) & M
    r2 = ((((p + r) & M) * 0x80000000) >> 32)
    a2 = ~(c2 | l2 | r2) & al & M
    plast = c2 >= thr
    pcnt = a2 != 0 and plast
    ppush = a2 != 0 and not plast
    if ar != 0 and ppush:
        stack[top] = (c, l, r, ar)
        top += 1
    if ar == 0 and not ppush:
        top -= 1
        assert top >= 0, "popped below the stack"
        c, l, r, av = stack[top]
    elif ppush:
        c, l, r, av = c2, l2, r2, a2
    else:
        av = ar
    return (c, l, r, av), top, 1 if pcnt else 0


def allowed_masks(n, queens):
    """Per-row allowed columns under the given queens (rows >= n and 31: none)."""
    last = (1 << n) - 1
    out = [0] * 32
    for row in range(n):
        m = last
        for qr, qc in queens:
            if qr == row:
                m &= 1 << qc
            else:
                for col in (qc, qc + (row - qr), qc - (row - qr)):
                    if 0 <= col < n:
                        m &= ~(1 << col)
        out[row] = m
    return out


def count_constrained_model(n, queens):
    """Whole board under the constraints from row 0 (one subproblem at d = 0),
    lane running whole 31-step rounds on two sentinel frames."""
    allowed = allowed_masks(n, queens)
    if n == 1:
        return 1 if allowed[0] else 0
    a0 = allowed[0]
    stack = {0: SENTINEL_C, 1: SENTINEL_C}
    state, top = (0, 0, 0, a0), 2
    thr = (n - 1) << ROW_SHIFT
    sol = 0
    while True:
        for _ in range(31):
            state, top, s = step_constrained(state, stack, top, allowed, thr)
            sol += s
            assert top <= n, "more than N - d slots"
        if top <= 1:
            return sol


@pytest.mark.parametrize("seed", range(3))
def test_constrained_model_equals_oracle(orc, seed):
    import synth_inputs
    g = synth_inputs.SplitMix64(900 + seed)
    for _ in range(6):
        n = 5 + g.below(5)        # 5..9
        qs = synth_inputs.constraint_set(g, n, g.below(4))
        assert count_constrained_model(n, qs) == orc.count_constrained(n, qs)[0], (n, qs)


def test_constrained_sentinel_lasts_a_round():
    allowed = [0] * 32
    stack = {0: SENTINEL_C, 1: SENTINEL_C}
    state, top = SENTINEL_C, 1
    for _ in range(31):
        state, top, s = step_constrained(state, stack, top, allowed, 5 << ROW_SHIFT)
        assert s == 0 and 0 <= top <= 1


# --- the avail-only stack (layout AVAIL) -----------------------------------------

def search_avail(rec, words):
    """One subproblem on the avail-only stack, the lane running whole 15-step
    rounds: columns at bits 1..N with guard columns pre-set, one word per level
    (the level's candidates with the chosen column in them, and the two bits
    the diagonal shifts drop), the parent state restored exactly by undoing the
    placement. Returns (solutions, nodes, deepest)."""
    n = (int(rec["meta"]) >> 2) & 31
    d = (int(rec["meta"]) >> 7) & 31
    last = (1 << n) - 1
    l0, r0 = int(rec["ld"]), int(rec["rd"]) & last
    c = ((int(rec["cols"]) << 1) | (~(last << 1) & M)) & M
    l, r = (l0 << 1) & M, (r0 << 1) & M
    av = ~(c | l | r) & M
    if d == n:
        return 1, 0, 0
    if d + 1 == n or av == 0:
        s = popc(av)
        return s, s, 0
    stack, top, sol, nodes, deepest = [], 0, 0, 0, 0
    while True:
        for _ in range(15):
            pv = av != 0
            p = av & ((av * M) & M)
            ar = (p * M + av) & M
            c2 = (p + c) & M
            l2 = (l * 2 + p * 2) & M
            r2 = ((((p + r) & M) * 0x80000000) >> 32)
            a2 = ~(c2 | l2 | r2) & M
            lastrow = popc(c2) == 31
            sol += 1 if (lastrow and a2) else 0
            nodes += 1 if pv else 0
            push = pv and not lastrow and a2 != 0
            if push:
                # the word: the candidates (p included) at bits 1..N, and in the
                # guard bits the one bit each shift drops: bit 0 of rd + p, bit 31
                # of ld + p
                lp, rp = (l + p) & M, (p + r) & M
                stack.append(av | (rp & 1) | (lp & 0x80000000))
                top += 1
                assert top <= words, "more words than the stack has"
                deepest = max(deepest, top)
                c, l, r, av = c2, l2, r2, a2
            elif ar == 0 and top > 0:
                top -= 1
                w = stack.pop()
                v = w & 0x7FFFFFFE
                q = v & ((v * M) & M)
                c = (c - q) & M
                l = ((((l * 0x80000000) >> 32) | (w & 0x80000000)) - q) & M
                r = (((r * 2) & M | (w & 1)) - q) & M
                av = (v - q) & M
            else:
                av = ar
        if top == 0 and av == 0:
            return sol, nodes + sol, deepest


@pytest.mark.parametrize("n,d", [(6, 2), (8, 3), (9, 4), (10, 3), (10, 6), (11, 5), (7, 7),
                                 (9, 8), (12, 4), (8, 1), (13, 2)])
def test_avail_only_model_equals_oracle(orc, n, d):
    pre = nq.enumerate_prefixes(n, d)
    cols, _ = orc.prefixes(n, d)
    want, want_nodes = orc.count_prefixes(n, cols)
    words = max(n - 2 - d, 1)
    for i, rec in enumerate(pre):
        sol, nodes, _ = search_avail(rec, words)
        assert (sol, nodes) == (int(want[i]), int(want_nodes[i])), (n, d, i)
