"""Pins of the CPU oracle to facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself:
  * values the paper prints (Tables 2 and 3, Appendix C; section 3.2's
    encoding example) -- tests/golden;
  * closed forms (l = 1, d = 2: 2/(sigma+1); (2,2,2): 8/11);
  * brute force: W_n computed from its definition by exhaustive enumeration
    and an LCS dynamic program (tests/bruteforce.py) -- the iterates must stay
    below it and F must map it below itself, tightly (Eqs. ineq1-ineq3);
  * invariants of F (Lemma 1: monotonicity, translation invariance; section
    3.3: complement symmetry) and of directed rounding.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import load_golden
import bruteforce as bf
import inputs


def floor6(x):
    return math.floor(x * 1e6 + 1e-9) / 1e6


def matches_printed(value, printed):
    """The paper prints 6 decimals, rounded down (Tables 2, 3) or to nearest (App. C)."""
    return abs(floor6(value) - printed) < 1e-9 or abs(round(value * 1e6) / 1e6 - printed) < 1e-9


# Appendix C cells that disagree with the paper's own other tables (see the
# design notes, readings of the paper):
#   (2,4,1), (2,5,1): printed 0.666666, but Table 3 gives 0.664722 (l = 6) and
#     0.639248 (l = 5) as the best bounds for d = 4, 5, which a 0.666666 at
#     l = 1 would contradict; the l = 1 column pairs d = 2k, 2k+1 with equal
#     values and the oracle gives 8/13 for both.
#   (3,6,1): printed 0.421434; Table 3 lists 0.421436 as the previous (Kiwi-Soto)
#     bound for (3,6), which the paper states it reproduces; the oracle gives
#     0.421436.
APPENDIX_C_EXCEPTIONS = {(2, 4, 1): 8 / 13, (2, 5, 1): 8 / 13, (3, 6, 1): 0.421436}


def iters_for(d):
    """Iteration count used for table pins (the paper never states n)."""
    return max(200, 100 * d)


def cost(s, d, h):
    return s ** (d * h) * s ** d * iters_for(d)


def table_cases(max_cost):
    seen = {}
    for row in load_golden("appendix_c.txt"):
        s, d, h = map(int, row[:3])
        seen[(s, d, h)] = ("Appendix C", float(row[3]))
    for row in load_golden("table3_general.txt"):
        s, d, h = map(int, row[:3])
        seen.setdefault((s, d, h), ("Table 3", float(row[3])))
    for row in load_golden("table2_binary.txt"):
        h = int(row[0])
        seen.setdefault((2, 2, h), ("Table 2", float(row[1])))
    return [(k, v) for k, v in sorted(seen.items()) if cost(*k) <= max_cost]


# ---------------------------------------------------------------------------
# section 3.2: the index


def test_encoding_example(orc):
    (s, d, h, a, b, idx), = load_golden("encoding_example.txt")
    s, d, h, idx = int(s), int(d), int(h), int(idx)
    digits = [[int(a[p]), int(b[p])] for p in range(h)]
    assert orc.encode(s, d, h, digits) == idx
    assert orc.strings_of(s, d, h, idx) == [tuple(map(int, a)), tuple(map(int, b))]


@pytest.mark.parametrize("s,d,h", [(2, 2, 3), (3, 2, 2), (2, 3, 2), (4, 2, 2)])
def test_encode_decode_roundtrip(orc, s, d, h):
    n = s ** (d * h)
    for x in range(n):
        assert orc.encode(s, d, h, orc.decode(s, d, h, x)) == x
        assert orc.strings_of(s, d, h, x) == bf.state_strings(s, d, h, x)


@pytest.mark.parametrize("h", [2, 3, 4])
def test_head_class_ranges(orc, h):
    """Section 3.2: [0, 2^(2h-2)) heads 00; up to 2^(2h-1)+2^(2h-2) unequal; rest 11."""
    for x in range(4 ** h):
        a, b = orc.strings_of(2, 2, h, x)
        if x < 2 ** (2 * h - 2):
            assert a[0] == b[0] == 0
        elif x < 2 ** (2 * h - 1) + 2 ** (2 * h - 2):
            assert a[0] != b[0]
        else:
            assert a[0] == b[0] == 1


@pytest.mark.parametrize("h", [2, 3])
def test_complement_index(orc, h):
    """Eq. impl:comp_eq: j = 2^(2h)-1-i holds the complemented pair."""
    n = 4 ** h
    for i in range(n // 2):
        a, b = orc.strings_of(2, 2, h, i)
        ca, cb = orc.strings_of(2, 2, h, n - 1 - i)
        assert ca == tuple(1 - c for c in a) and cb == tuple(1 - c for c in b)


# ---------------------------------------------------------------------------
# printed bounds and closed forms


@pytest.mark.parametrize("arith", ["fx", "f64"])
@pytest.mark.parametrize("sigma", range(2, 11))
def test_closed_form_l1_d2(orc, sigma, arith):
    """App. C, l = 1, d = 2 row: 2/(sigma+1)."""
    res = orc.run(sigma, 2, 1, 200, arith=arith)
    assert abs(res["bound_rd"] - 2 / (sigma + 1)) < 1e-9
    assert res["bound_rd"] <= 2 / (sigma + 1) + 1e-15


@pytest.mark.parametrize("arith", ["fx", "f64"])
def test_closed_form_8_over_11(orc, arith):
    """Table 2 / App. C: (2,2,2) is 0.727272 / 0.727273, i.e. 8/11."""
    res = orc.run(2, 2, 2, 200, arith=arith)
    assert abs(res["bound_rd"] - 8 / 11) < 1e-9


@pytest.mark.parametrize("key,src", table_cases(max_cost=4e7), ids=lambda v: str(v))
def test_printed_bounds(orc, key, src):
    s, d, h = key
    where, printed = src
    res = orc.run(s, d, h, iters_for(d), arith="fx")
    b = res["bound_rd"]
    if key in APPENDIX_C_EXCEPTIONS:
        assert abs(b - APPENDIX_C_EXCEPTIONS[key]) < 1e-6
        return
    if where != "Appendix C":
        assert abs(floor6(b) - printed) < 1e-9, (where, b, printed)
    else:
        assert matches_printed(b, printed), (where, b, printed)


def test_printed_bounds_f64_agree(orc):
    for key, (where, printed) in table_cases(max_cost=2e6):
        if key in APPENDIX_C_EXCEPTIONS:
            continue
        s, d, h = key
        b = orc.run(s, d, h, iters_for(d), arith="f64")["bound_rd"]
        assert matches_printed(b, printed), (key, b, printed)


def test_binary_bounds_increase_with_h_and_stay_below_upper_bound(orc):
    """Table 2 increases with l; every lower bound is below Lueker's upper bound 0.826280 (abstract)."""
    prev = 0.0
    for h in range(1, 7):
        b = orc.run(2, 2, h, 200, arith="fx")["bound_rd"]
        assert prev < b < 0.826280
        prev = b


# ---------------------------------------------------------------------------
# brute force: W_n from its definition


BRUTE = [(2, 2, 2, 4), (2, 2, 1, 6), (2, 3, 1, 3), (3, 2, 1, 3)]


@pytest.fixture(scope="module")
def brute_tables():
    return {c: bf.W_table(*c) for c in BRUTE}


@pytest.mark.parametrize("case", BRUTE)
def test_F_of_W_below_W_and_tight(orc, brute_tables, case):
    """Eqs. ineq1-ineq3: W_n >= F(W_{n-1}, .., W_{n-d}) at every state, with equality somewhere."""
    s, d, h, nm = case
    W = brute_tables[case]
    N = s ** (d * h)
    for n in range(d, nm + 1):
        if s == 2:  # dyadic values: f64 evaluates F exactly
            vs = [np.array([float(W[n - k][x]) for x in range(N)]) for k in range(1, d + 1)]
            Fv = orc.F(s, d, h, vs, arith="f64")
            Wn = np.array([float(w) for w in W[n]])
            assert np.all(Fv <= Wn)
            assert np.any(Fv == Wn)
        else:  # F in fixed point rounds down: a pin from below within 2^-K per mean
            K = 44
            vs = [np.array([math.floor(W[n - k][x] * (1 << K)) for x in range(N)], dtype=np.int64)
                  for k in range(1, d + 1)]
            Fv = orc.F(s, d, h, vs, arith="fx")
            for x in range(N):
                assert Fraction(int(Fv[x]), 1 << K) <= W[n][x]
            gap = min(W[n][x] - Fraction(int(Fv[x]), 1 << K) for x in range(N))
            assert gap < Fraction(4, 1 << K)


@pytest.mark.parametrize("case", BRUTE)
@pytest.mark.parametrize("arith", ["fx", "f64"])
def test_iterates_below_W(orc, brute_tables, case, arith):
    """Zero-start iterates are lower bounds: v_n <= W_n (section 2.1)."""
    s, d, h, nm = case
    W = brute_tables[case]
    N = s ** (d * h)
    for n in range(d, nm + 1):
        res = orc.run(s, d, h, n - d + 1, arith=arith)
        v = res["iterates"][0]
        for x in range(N):
            val = Fraction(int(v[x]), 1 << 44) if arith == "fx" else Fraction(float(v[x]))
            assert val <= W[n][x] + Fraction(1, 10 ** 12)


@pytest.mark.parametrize("case", [c for c in BRUTE if c[1] <= 3])
def test_all_subsets_F_between_F_and_W(orc, brute_tables, case):
    """f_mode 1 (every non-empty advance set, +1 on the full set for equal
    heads): each candidate drops the heads of some strings, a move that can
    only lower the LCS, so F_all(W) <= W; its candidates include every N_z of
    Alg. 1, so F(W) <= F_all(W); hence equality wherever F(W) = W."""
    s, d, h, nm = case
    W = brute_tables[case]
    N = s ** (d * h)
    K = 44
    for n in range(d, nm + 1):
        vs = [np.array([math.floor(W[n - k][x] * (1 << K)) for x in range(N)], dtype=np.int64)
              for k in range(1, d + 1)]
        F0 = orc.F(s, d, h, vs, arith="fx")
        F1 = orc.F(s, d, h, vs, arith="fx", f_mode=1)
        assert np.all(F1 >= F0)
        for x in range(N):
            assert Fraction(int(F1[x]), 1 << K) <= W[n][x]
        assert min(W[n][x] - Fraction(int(F1[x]), 1 << K) for x in range(N)) < Fraction(4, 1 << K)


@pytest.mark.parametrize("case", [c for c in BRUTE if c[1] <= 3])
def test_all_subsets_iterates_below_W(orc, brute_tables, case):
    s, d, h, nm = case
    W = brute_tables[case]
    for n in range(d, nm + 1):
        v = orc.run(s, d, h, n - d + 1, f_mode=1)["iterates"][0]
        v0 = orc.run(s, d, h, n - d + 1)["iterates"][0]
        assert np.all(v >= v0)
        for x in range(s ** (d * h)):
            assert Fraction(int(v[x]), 1 << 44) <= W[n][x]


# Values of the all-advance-sets F (f_mode 1) worked out by hand at single
# states, one for each kind of set that can win the max.  f_mode 1 is the max,
# over every non-empty set N of strings, of the mean over the appended letters
# of v_|N| at the state whose strings in N lose their head and gain the letter
# at their end; when every head is equal the full set carries the +1 of the
# match (the extension of Algorithm 1 and Eq. ineq3 that reading R15 takes).
# The paper's F (f_mode 0) only has the sets N_z = {j : head_j != z}.  With
# h = 1 a state is one letter per string, and a string that advances becomes
# the appended letter.  Values are in units; every one is exact in fixed point
# and in binary floating point.
def _unit_vector(n, where, value):
    v = np.zeros(n)
    for x in where:
        v[x] = value
    return v


def all_subsets_hand_worked_cases():
    """(name, (s, d, h), arguments v_1..v_d, state, F_all at the state, F at the state)."""
    cases = []
    # (2,3,1), state (a,b,c) = (0,0,1), index 0*4 + 0*2 + 1 = 1: heads 0,0,1.
    # N_0 = {c} and N_1 = {a,b}; the other five sets are extra.
    # A: v_1 = 8 at (1,0,1) (index 5), v_2 = v_3 = 0.  Advancing a alone
    #    reads v_1 at (0,0,1) and (1,0,1): (0 + 8)/2 = 4.  Every other set reads
    #    only zeros: {c} reads (0,0,0), (0,0,1); {b} reads (0,0,1), (0,1,1);
    #    the pairs and the full set read v_2, v_3.  So F_all = 4, won by a
    #    singleton of a majority string; F (unequal heads, no +1) = 0.
    cases.append(("majority singleton", (2, 3, 1), [_unit_vector(8, [5], 8.0), np.zeros(8), np.zeros(8)], 1, 4.0, 0.0))
    # B: v_2 = 8 at (1,0,0) (index 4), v_1 = v_3 = 0.  Advancing {a, c} reads
    #    v_2 at (x,0,z) for x, z in {0,1}: indices 0, 1, 4, 5 -> (0+0+8+0)/4 = 2.
    #    {a,b} reads (x,y,1): 1, 3, 5, 7 -> 0; {b,c} reads (0,y,z): 0..3 -> 0;
    #    singletons read v_1 = 0, the full set v_3 = 0.  F_all = 2, won by a pair
    #    holding the minority string; F = max({c}: 0, {a,b}: 0) = 0.
    cases.append(("pair with the minority", (2, 3, 1), [np.zeros(8), _unit_vector(8, [4], 8.0), np.zeros(8)], 1, 2.0, 0.0))
    # C: v_3 = 8 everywhere, v_1 = v_2 = 0.  The full set's mean is 8 and gets
    #    no +1 (the heads differ); every other set reads zeros.  F_all = 8, F = 0.
    cases.append(("full set, unequal heads", (2, 3, 1), [np.zeros(8), np.zeros(8), np.full(8, 8.0)], 1, 8.0, 0.0))
    # E: (2,2,1), state (0,0), index 0: equal heads.  v_1 = 0, v_2 = 5
    #    everywhere.  The full set gives 1 + 5 = 6 (the match), {a} and {b}
    #    read v_1: 0.  F_all = 6 = F.
    cases.append(("full set with the match", (2, 2, 1), [np.zeros(4), np.full(4, 5.0)], 0, 6.0, 6.0))
    return cases


# D, on the exact W tables: (2,2,2), strings a = 00, b = 01 (index 1: the
# digits a_0 b_0 a_1 b_1 = 0 0 0 1), n = 2, so the arguments are v_1 = W_1 and
# v_2 = W_0.  W_0 is the LCS of the two strings themselves; W_1 adds one
# random letter to the string of our choice, after seeing the letters.
#  * The match (full set, +1): 1 + the mean of W_0 over (0c, 1e): LCS(00, 10)
#    = 1, LCS(00, 11) = 0, LCS(01, 10) = 1, LCS(01, 11) = 1 -> 1 + 3/4 = 7/4.
#    That is the paper's F here (both heads are 0, so N_1 is the full set).
#  * Advancing a alone: the mean of W_1 at (00, 01) and (01, 01).
#    W_1(01, 01) = 2: the LCS is already 2 and cannot exceed the length 2 of
#    the string left alone.  W_1(00, 01): the LCS is 1; a letter x for a and y
#    for b are drawn, and appending x = 1 to a (001 vs 01) or y = 0 to b (00
#    vs 010) reaches 2, which fails only when x = 0 and y = 1: 3/4 * 2 + 1/4 *
#    1 = 7/4.  The mean is (7/4 + 2)/2 = 15/8.
#  * Advancing b alone: the mean of W_1 at (00, 10) and (00, 11): at most
#    (7/4 + 1)/2 < 15/8 (each LCS is at most 1, plus 1 with a drawn letter).
# So F_all(W_1, W_0) = 15/8, won by a proper subset that skips the match, and
# F(W_1, W_0) = 7/4.
HAND_D = dict(shape=(2, 2, 2), state=1, W1={("00", "01"): Fraction(7, 4), ("01", "01"): Fraction(2)},
              F_all=Fraction(15, 8), F=Fraction(7, 4))


def _bits_state(a, b):
    """index of (a, b) for sigma = d = 2, h = 2: digits a_0 b_0 a_1 b_1"""
    return a[0] * 8 + b[0] * 4 + a[1] * 2 + b[1]


def all_subsets_hand_worked_failures(orc, W222=None):
    """the hand-worked f_mode 1 values that the oracle misses (empty: all agree)"""
    failures = []
    K = 44
    for name, (s, d, h), vs, x, want_all, want_f in all_subsets_hand_worked_cases():
        for arith in ("fx", "f64"):
            args = [np.array([int(val * (1 << K)) for val in v], dtype=np.int64) for v in vs] if arith == "fx" else vs
            scale = (1 << K) if arith == "fx" else 1
            got_all = orc.F(s, d, h, args, arith=arith, f_mode=1)[x]
            got_f = orc.F(s, d, h, args, arith=arith)[x]
            if got_all != want_all * scale or got_f != want_f * scale:
                failures.append(f"{name} ({arith})")
    W = W222 if W222 is not None else bf.W_table(2, 2, 2, 2)
    for (a, b), val in HAND_D["W1"].items():  # the hand-worked W_1 values are the brute force's
        assert W[1][_bits_state([int(c) for c in a], [int(c) for c in b])] == val
    vs = [np.array([int(W[1][y] * (1 << K)) for y in range(16)], dtype=np.int64),
          np.array([int(W[0][y] * (1 << K)) for y in range(16)], dtype=np.int64)]
    x = HAND_D["state"]
    if (orc.F(2, 2, 2, vs, arith="fx", f_mode=1)[x] != HAND_D["F_all"] * (1 << K)
            or orc.F(2, 2, 2, vs, arith="fx")[x] != HAND_D["F"] * (1 << K)):
        failures.append("proper subset beats the match on W")
    return failures


def test_all_subsets_hand_worked(orc, brute_tables):
    """f_mode 1 equals the values worked out by hand, one state per kind of winning set."""
    assert all_subsets_hand_worked_failures(orc, brute_tables[(2, 2, 2, 4)]) == []


def test_all_subsets_adds_candidates():
    """On random arguments the extra advance sets win somewhere (the test above is not vacuous)."""
    import oracle as orc_mod

    rng = np.random.default_rng(5)
    for s, d, h in [(2, 2, 3), (2, 3, 2), (3, 2, 2)]:
        N = s ** (d * h)
        vs = [rng.integers(-(1 << 46), 1 << 46, size=N, dtype=np.int64) for _ in range(d)]
        F0 = orc_mod.F(s, d, h, vs, arith="fx")
        F1 = orc_mod.F(s, d, h, vs, arith="fx", f_mode=1)
        assert np.all(F1 >= F0) and np.any(F1 > F0)


# ---------------------------------------------------------------------------
# invariants of F and of the iteration


SHAPES = [(2, 2, 3), (3, 2, 2), (2, 3, 2), (4, 2, 1), (2, 4, 1)]


@pytest.mark.parametrize("s,d,h", SHAPES)
def test_translation_invariance_exact(orc, s, d, h):
    """Lemma 1's second property: F(v + c) = F(v) + c exactly (fx: any c; f64: dyadic c, exact sums)."""
    vs = inputs.random_history(s, d, h, seed=11)
    F0 = orc.F(s, d, h, vs, arith="fx")
    c = 12345678901 + (1 << 44) * 3
    F1 = orc.F(s, d, h, [v + c for v in vs], arith="fx")
    assert np.array_equal(F1, F0 + c)
    small = [np.floor(v / 2.0 ** 40) / 16.0 for v in vs]  # dyadic values, exact sums
    G0 = orc.F(s, d, h, small, arith="f64")
    G1 = orc.F(s, d, h, [v + 0.75 for v in small], arith="f64")
    assert np.array_equal(G1, G0 + 0.75)


@pytest.mark.parametrize("s,d,h", SHAPES)
def test_monotonicity(orc, s, d, h):
    """Lemma 1's first property: v <= v' componentwise implies F(v) <= F(v')."""
    rng = np.random.default_rng(5)
    vs = inputs.random_history(s, d, h, seed=3)
    bumped = [v + rng.integers(0, 1 << 40, size=v.size, dtype=np.int64) for v in vs]
    assert np.all(orc.F(s, d, h, bumped, arith="fx") >= orc.F(s, d, h, vs, arith="fx"))
    f = [v.astype(np.float64) / 2.0 ** 44 for v in vs]
    fb = [v.astype(np.float64) / 2.0 ** 44 for v in bumped]
    assert np.all(orc.F(s, d, h, fb, arith="f64") >= orc.F(s, d, h, f, arith="f64"))


@pytest.mark.parametrize("d,h", [(2, 3), (3, 2), (4, 1)])
def test_complement_symmetry_fx(orc, d, h):
    """Section 3.3: complementing every string leaves v unchanged -- exact in fixed point."""
    n = 2 ** (d * h)
    flip = inputs.complement_index(n)
    res = orc.run(2, d, h, 60, arith="fx")
    for v in res["iterates"]:
        assert np.array_equal(v, v[flip])
    vs = inputs.random_history(2, d, h, seed=9)
    assert np.array_equal(orc.F(2, d, h, [v[flip] for v in vs], arith="fx"), orc.F(2, d, h, vs, arith="fx")[flip])


def test_string_swap_symmetry_fx(orc):
    """LCS is symmetric in its arguments: swapping the two strings leaves the fx iterate unchanged."""
    s, d, h = 3, 2, 2
    n = s ** (d * h)
    swap = np.array([orc.encode(s, d, h, orc.decode(s, d, h, x)[:, ::-1]) for x in range(n)])
    res = orc.run(s, d, h, 50, arith="fx")
    v = res["iterates"][0]
    assert np.array_equal(v, v[swap])


@pytest.mark.parametrize("s,d,h", [(2, 2, 3), (3, 2, 2), (2, 3, 2)])
def test_zero_start_iterates_nondecreasing(orc, s, d, h):
    res = orc.run(s, d, h, 30, arith="fx")
    it = res["iterates"]
    for k in range(d - 1):
        assert np.all(it[k] >= it[k + 1])


@pytest.mark.parametrize("s,d,h", [(2, 2, 4), (3, 2, 2), (2, 3, 2)])
def test_fx_tracks_f64(orc, s, d, h):
    """The two arithmetics differ only by rounding: relative 1e-12 after 300 iterations."""
    a = orc.run(s, d, h, 300, arith="fx")
    b = orc.run(s, d, h, 300, arith="f64")
    va = a["iterates"][0].astype(np.float64) / 2.0 ** 44
    vb = b["iterates"][0]
    assert np.max(np.abs(va - vb) / np.abs(vb)) < 1e-12
    assert abs(a["bound_rd"] - b["bound_rd"]) < 1e-10


@pytest.mark.parametrize("s,d,h", [(2, 2, 3), (3, 2, 2), (2, 3, 2)])
def test_kept_triplet_is_feasible(orc, s, d, h):
    """Lemma 1's third condition for the returned (u, r, eps): F(u+(d-1)r, .., u) >= u + (dr - eps)."""
    res = orc.run(s, d, h, 120, arith="fx", check_every=10, want_u=True)
    u, r, eps = res["u"], res["r"], res["eps"]
    assert 0 <= eps <= r
    args = [u + (d - k) * r for k in range(1, d + 1)]
    Fv = orc.F(s, d, h, args, arith="fx")
    assert np.all(Fv >= u + d * r - eps)
    assert np.any(Fv == u + d * r - eps) or eps == 0  # eps is the least such value (or clipped at 0)


@pytest.mark.parametrize("s,d,h", [(2, 2, 3), (3, 2, 2)])
def test_check_matches_lemma(orc, s, d, h):
    """E from the check is the least eps >= 0 making (u, R, eps) feasible."""
    vs = inputs.random_history(s, d, h, seed=21)
    u = vs[0]
    R = int(0.4 * (1 << 44))
    E, W = orc.check(s, d, h, u, R, arith="fx", want_W=True)
    args = [u + (d - k) * R for k in range(1, d + 1)]
    Fv = orc.F(s, d, h, args, arith="fx")
    assert np.array_equal(W, u + d * R - Fv)
    assert E == max(0, int(W.max()))


def test_r_mode_max_gives_same_converged_bound(orc):
    """Algorithm 2 as printed takes R = max increment; the bound converges to the same value."""
    a = orc.run(2, 2, 4, 200, arith="fx", r_mode=0)
    b = orc.run(2, 2, 4, 200, arith="fx", r_mode=1)
    assert abs(a["bound_rd"] - b["bound_rd"]) < 1e-9


def test_argmin_is_a_minimiser(orc):
    s, d, h = 2, 2, 4
    res = orc.run(s, d, h, 37, arith="fx")
    v0, v1 = res["iterates"][0], res["iterates"][1]
    inc = v0 - v1
    assert inc.min() == res["R"]
    assert res["argmin"] == int(np.argmin(inc))


# ---------------------------------------------------------------------------
# directed rounding


def test_directed_rounding_helpers(orc):
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a = float(rng.normal() * 10.0 ** int(rng.integers(-5, 5)))
        b = float(rng.normal() * 10.0 ** int(rng.integers(-5, 5)))
        exact = Fraction(a) + Fraction(b)
        lo, hi = orc.add_dir(a, b, orc.RD), orc.add_dir(a, b, orc.RU)
        assert Fraction(lo) <= exact <= Fraction(hi)
        assert lo == hi or math.nextafter(lo, math.inf) == hi
        k = float(rng.integers(1, 9))
        exact = Fraction(k) * Fraction(a)
        lo, hi = orc.mul_dir(k, a, orc.RD), orc.mul_dir(k, a, orc.RU)
        assert Fraction(lo) <= exact <= Fraction(hi)
        m = float(3 ** rng.integers(1, 6))
        exact = Fraction(a) / Fraction(m)
        lo, hi = orc.div_dir(a, m, orc.RD), orc.div_dir(a, m, orc.RU)
        assert Fraction(lo) <= exact <= Fraction(hi)
        assert lo == hi or math.nextafter(lo, math.inf) == hi


def test_fx_to_double_rounds_down(orc):
    for a in [0, 1, -1, (1 << 53) + 1, -(1 << 53) - 1, (1 << 62) + 12345, -(1 << 62) - 3]:
        x = orc.fx_to_double_rd(a, 0)
        assert Fraction(x) <= a and Fraction(math.nextafter(x, math.inf)) > a


def _run_arith(arith):
    import oracle

    res = oracle.run(2, 2, 8, 2000, arith=arith, check_every=0)
    return res["iterates"][0], res["bound_rd"]


def test_fx_tracks_f64_at_config_size():
    """The GPU path computes in int64 fixed point (44 fractional bits, floor
    means) and equals the oracle's fx mode bit for bit; the benchmark spec's
    tolerance is stated against FP64.  At the config size (2,2,8) and its 2000
    iterations, where the floor drift T 2^-44 is largest, the fx iterate stays
    within 1e-12 relative of the f64 one (round to nearest, R5's order), the
    two bounds agree to 1e-12, and both floor to Table 2's 0.776860."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(2) as pool:  # the two arithmetics side by side
        (v_fx, b_fx), (v_64, b_64) = pool.map(_run_arith, ["fx", "f64"])
    v = v_fx.astype(np.float64) / (1 << 44)  # exact: |v| < 2^10, so fx values have < 53 significant bits
    T = 2000
    assert np.max(np.abs(v - v_64) / np.abs(v_64)) <= 1e-12
    assert np.max(np.abs(v - v_64)) <= T * 2.0 ** -44 + T * 4 * np.finfo(np.float64).eps * np.max(np.abs(v_64))
    assert abs(b_fx - b_64) <= 1e-12
    assert floor6(b_fx) == floor6(b_64) == 0.776860
