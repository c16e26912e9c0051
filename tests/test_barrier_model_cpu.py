"""Model check, on CPU, of the grid barrier's overflow flag.

After a grid level every CTA measures the pairs it discovered from its own
shared-memory buffer; a CTA whose buffer overflowed raises a flag in the
barrier word as it arrives, and when the barrier reports the flag the whole
grid measures the level again from the lists between two more barriers,
after which CTA 0 clears the flag.  The traversal kernel's barrier word
holds the generation and the flag bits; here the same protocol is restated
as small state machines (one per CTA, one shared word, one arrival counter)
and every interleaving of their shared-memory steps is explored.

The property: at every level all CTAs take the same branch (re-measure or
not), that branch is right (some CTA overflowed at that level), and every
CTA finishes (no barrier left waiting).  The kernel's rule, one of two bits
chosen by the parity of the generation the barrier closes and cleared only
after the next barrier, satisfies it; a single bit, or a flag cleared right
after the barrier that reported it, does not (a CTA still waiting in the
barrier can then read a flag meant for the next one, or miss its own)."""

import itertools

import pytest

PARITY, SINGLE, SINGLE_EARLY_CLEAR = "parity", "single", "single_early_clear"
N_LEVELS = 3


def flag_bit(rule, gen):
    return 1 << (gen & 1) if rule == PARITY else 1


def next_level(lv, res):
    return (lv + 1, "done" if lv + 1 == N_LEVELS else "enter", 0, "L", res)


def after_barrier(i, lv, which, r, res, rule):
    """A CTA's state once it has left barrier `which` of level lv: "L" ends
    the level (r: the flag it read), "B" and "C" bracket the re-measurement
    from the lists; CTA 0 clears the flag after B (or, in the faulty
    variant, right after L)."""
    if which == "L":
        res = res + (r,)
        if not r:
            return next_level(lv, res)
        if rule == SINGLE_EARLY_CLEAR and i == 0:
            return (lv, "clear", 0, "B", res)
        return (lv, "enter", 0, "B", res)
    if which == "B":
        if i == 0 and rule != SINGLE_EARLY_CLEAR:
            return (lv, "clear", 0, "C", res)
        return (lv, "enter", 0, "C", res)
    return next_level(lv, res)


def explore(rule, n_ctas, flags):
    """flags[i][lv]: CTA i's buffer overflows at level lv.  Explores every
    interleaving; returns the first violation found (a string) or None."""
    truth = tuple(any(flags[i][lv] for i in range(n_ctas)) for lv in range(N_LEVELS))
    # shared: arrival count, generation, flag bits; per CTA: (level, phase,
    # generation read on entering the barrier, which barrier, branches taken)
    init = (0, 0, 0, tuple((0, "enter", 0, "L", ()) for _ in range(n_ctas)))
    seen, stack = set(), [init]
    while stack:
        state = stack.pop()
        if state in seen:
            continue
        seen.add(state)
        count, gen, bits, ctas = state
        if all(c[1] == "done" for c in ctas):
            for i, c in enumerate(ctas):
                if c[4] != truth:
                    return f"CTA {i} took {c[4]}, the levels' flags were {truth}"
            continue
        moves = []
        for i, (lv, ph, g, which, res) in enumerate(ctas):
            shared, me = (count, gen, bits), None
            if ph == "enter":  # read the generation this barrier closes
                me = (lv, "flag" if which == "L" else "arrive", gen, which, res)
            elif ph == "flag":  # raise the flag for that generation
                if flags[i][lv]:
                    shared = (count, gen, bits | flag_bit(rule, g))
                me = (lv, "arrive", g, which, res)
            elif ph == "arrive":
                if count == n_ctas - 1:  # the last arrival opens the barrier
                    shared = (0, gen + 1, bits)
                    me = after_barrier(i, lv, which, bool(bits & flag_bit(rule, g)), res, rule)
                else:
                    shared = (count + 1, gen, bits)
                    me = (lv, "wait", g, which, res)
            elif ph == "wait" and gen != g:  # the read that ends the wait
                me = after_barrier(i, lv, which, bool(bits & flag_bit(rule, g)), res, rule)
            elif ph == "clear":  # CTA 0 clears every flag bit
                shared = (count, gen, 0)
                me = (lv, "enter", 0, which, res)
            if me is not None:
                moves.append(shared + (ctas[:i] + (me,) + ctas[i + 1:],))
        if not moves:
            return f"barrier never completes: {ctas}"
        stack.extend(moves)
    return None


def scenarios(n_ctas):
    for b in itertools.product((0, 1), repeat=n_ctas * N_LEVELS):
        yield [list(b[i * N_LEVELS:(i + 1) * N_LEVELS]) for i in range(n_ctas)]


@pytest.mark.parametrize("n_ctas", [2, 3])
def test_parity_bits_hold_in_every_interleaving(n_ctas):
    for flags in scenarios(n_ctas):
        assert explore(PARITY, n_ctas, flags) is None, flags


def test_single_bit_lets_a_waiting_cta_take_the_next_levels_flag():
    # CTA 1 may still wait in level 0's barrier when CTA 0 flags level 1
    assert explore(SINGLE, 2, [[0, 1, 0], [0, 0, 0]]) is not None


def test_clearing_right_after_the_barrier_lets_a_waiting_cta_miss_the_flag():
    assert explore(SINGLE_EARLY_CLEAR, 2, [[1, 0, 0], [0, 0, 0]]) is not None


def test_model_without_flags_needs_no_remeasure():
    for rule in (PARITY, SINGLE, SINGLE_EARLY_CLEAR):
        assert explore(rule, 3, [[0] * N_LEVELS] * 3) is None
