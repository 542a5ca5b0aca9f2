"""Mutation test of the oracle's pins: every planted mistake must fail a pin.

The oracle source has compile-time hooks (ORC_MUTANT = k) that plant one
plausible mistake each -- a wrong shift direction, the arguments of F in
reverse order, the wrong divisor, min instead of max, a dropped +1, a flipped
increment, a check without the (d-k) R shift, transposed strings in the
index.  The pins below are the same facts test_oracle_pins.py uses (printed
values, closed forms, brute force, the encoding example); a mutant that passes
all of them would mean the pins cannot see that mistake.
"""
import math

import numpy as np
import pytest

from conftest import load_golden
import bruteforce as bf

MUTANTS = {
    1: "characters appended at the head instead of the end",
    2: "F reads its arguments in reverse order",
    3: "every mean divides by sigma^d",
    4: "min over z instead of max",
    5: "the +1 of equal heads dropped",
    6: "increment taken as v_{t-1} - v_t",
    7: "check evaluates F(u, .., u) without the (d-k) R shift",
    8: "strings transposed inside each position of the index",
}


def _pins_hold(orc):
    failures = []
    (s, d, h, a, b, idx), = load_golden("encoding_example.txt")
    digits = [[int(a[p]), int(b[p])] for p in range(int(h))]
    if orc.encode(int(s), int(d), int(h), digits) != int(idx):
        failures.append("encoding example")
    for x in range(16):
        if orc.encode(2, 2, 2, orc.decode(2, 2, 2, x)) != x:
            failures.append("encode/decode")
            break
    for sigma in (2, 3, 5):
        try:
            bd = orc.run(sigma, 2, 1, 200, arith="fx")["bound_rd"]
        except Exception:
            bd = float("nan")
        if not abs(bd - 2 / (sigma + 1)) < 1e-9:
            failures.append(f"closed form sigma={sigma}")
    for (s, d, h, val) in [(2, 2, 3, 0.747922), (3, 2, 2, 0.620690), (2, 3, 2, 0.673913)]:
        try:
            bd = orc.run(s, d, h, 300, arith="fx")["bound_rd"]
        except Exception:
            bd = float("nan")
        if not abs(math.floor(bd * 1e6 + 1e-9) / 1e6 - val) < 1e-9 and not abs(round(bd * 1e6) / 1e6 - val) < 1e-9:
            failures.append(f"table {s, d, h}")
    W = bf.W_table(2, 2, 2, 4)
    for n in range(2, 5):
        vs = [np.array([float(W[n - k][x]) for x in range(16)]) for k in (1, 2)]
        Fv = orc.F(2, 2, 2, vs, arith="f64")
        Wn = np.array([float(w) for w in W[n]])
        if not (np.all(Fv <= Wn) and np.any(Fv == Wn)):
            failures.append(f"brute force n={n}")
    return failures


def test_unmutated_oracle_passes(orc):
    assert _pins_hold(orc) == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda m: MUTANTS[m])
def test_mutant_is_caught(orc, mutant):
    with orc.use_mutant(mutant):
        failures = _pins_hold(orc)
    assert failures, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"


# mistakes in the generated arguments of the full-size GPU parity tests
GENERATED_MUTANTS = {
    9: "the d = 3 canonical index misses the complements of the permuted states",
    10: "the sigma = d = 2 canonical index misses the swapped complement",
    11: "SplitMix64 with a wrong finaliser shift",
}


def _generated_pins_hold(orc):
    import test_oracle_generated as gen

    failures = []
    for seed, i, out in load_golden("splitmix64_seed0.txt"):
        if orc.splitmix64_at(int(seed), int(i)) != int(out, 16):
            failures.append("SplitMix64 published outputs")
            break
    for s, d, h, sym in [(2, 2, 3, 2), (2, 3, 2, 3)]:
        vs, _ = gen._explicit(orc, s, d, h, sym)
        xs = np.arange(s ** (d * h), dtype=np.uint64)
        got = orc.F_generated(s, d, h, gen.SEEDS[:d], gen.BASES[:d], gen.SPREAD, xs, symmetric=sym)
        if not np.array_equal(got, orc.F(s, d, h, vs, arith="fx")):
            failures.append(f"generated arguments {s, d, h, sym}")
    return failures


def test_unmutated_generator_passes(orc):
    assert _generated_pins_hold(orc) == []


@pytest.mark.parametrize("mutant", sorted(GENERATED_MUTANTS), ids=lambda m: GENERATED_MUTANTS[m])
def test_generated_input_mutant_is_caught(orc, mutant):
    with orc.use_mutant(mutant):
        failures = _generated_pins_hold(orc)
    assert failures, f"mutant {mutant} ({GENERATED_MUTANTS[mutant]}) passed every pin"


# mistakes in the all-advance-sets F (f_mode 1), an extension the paper does
# not print values for; its pins are the hand-worked single-state values
F_MODE1_MUTANTS = {
    12: "f_mode 1 keeps only the sets N_z and the full set",
    13: "f_mode 1 never takes the full set",
    14: "f_mode 1 drops the +1 of the full set for equal heads",
    15: "f_mode 1 adds the +1 to every set when the heads are equal",
}


def _all_subsets_pins_hold(orc):
    import test_oracle_pins as pins

    return pins.all_subsets_hand_worked_failures(orc)


def test_unmutated_all_subsets_passes(orc):
    assert _all_subsets_pins_hold(orc) == []


@pytest.mark.parametrize("mutant", sorted(F_MODE1_MUTANTS), ids=lambda m: F_MODE1_MUTANTS[m])
def test_all_subsets_mutant_is_caught(orc, mutant):
    with orc.use_mutant(mutant):
        failures = _all_subsets_pins_hold(orc)
    assert failures, f"mutant {mutant} ({F_MODE1_MUTANTS[mutant]}) passed every pin"


@pytest.mark.parametrize("mutant", sorted(F_MODE1_MUTANTS), ids=lambda m: F_MODE1_MUTANTS[m])
def test_all_subsets_mutant_leaves_the_paper_F_alone(orc, mutant):
    """the f_mode 1 mutants change nothing of the paper's F: the f_mode 0 pins still hold"""
    with orc.use_mutant(mutant):
        assert _pins_hold(orc) == []
