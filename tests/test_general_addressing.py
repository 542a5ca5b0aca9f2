"""The general kernels' index arithmetic (sweep_rt.cuh), restated with plain
integers and checked against the terms that Algorithm 1 / Eq. ineq3 define,
written from the STATE INDEX definition of include/lcs_bound.h alone.

For a state with heads H and tails t_j, the candidate of letter z sums
v_{t-k} over the states in which each string j with H_j = z (the set S) keeps
z t_j and each other string (N, k = |N| of them) becomes t_j c_j, for every
c in Sigma^k.  The kernels form those states' indices from the tail's digit
parts: one range of terms per thread (or 32 contiguous chunks per warp, or
256 per CTA for entries of 2048 terms or more) for
every sigma, and, for sigma = 2 from d = 9 on, lane bits deposited into the
five lowest offset bits plus a submask walk over the rest.  Each must produce
every term once (as a multiset), for every state and every letter.  The GPU
parity tests compare the kernels' values with the oracle at 15 shapes; these
checks reach d = 16 and sigma = 10 on the CPU.
"""
import itertools

import numpy as np
import pytest

K_RT_TABLE = 6000
K_RT_WARP_D = 9


def state_index(strings, s, h):
    """The header's definition: digit p (0 = head) of string j weighs
    s^(d (h-1-p) + (d-1-j))."""
    d = len(strings)
    return sum(strings[j][p] * s ** (d * (h - 1 - p) + (d - 1 - j)) for j in range(d) for p in range(h))


def decode(x, s, d, h):
    """Inverse of state_index: the d strings of state x."""
    strings = [[0] * h for _ in range(d)]
    for p in range(h):
        for j in range(d):
            strings[j][p] = (x // s ** (d * (h - 1 - p) + (d - 1 - j))) % s
    return strings


def defined_terms(strings, z, s):
    """The states the candidate of letter z sums over (Algorithm 1, Eq. ineq3)."""
    d, h = len(strings), len(strings[0])
    S = [j for j in range(d) if strings[j][0] == z]
    N = [j for j in range(d) if j not in S]
    out = []
    for c in itertools.product(range(s), repeat=len(N)):
        nxt = [list(st) for st in strings]
        for i, j in enumerate(N):
            nxt[j] = strings[j][1:] + [c[i]]
        out.append(state_index(nxt, s, h))
    return sorted(out), len(N)


# --- the kernel's arithmetic, restated ------------------------------------

def rt_d_of(n_stored, s, h):
    dh, m = 0, n_stored
    while m > 1:
        m //= s
        dh += 1
    return dh // h


def tail_parts(t, s, d, h):
    tp, w = [0] * d, 1
    for q in range(d * (h - 1)):
        tp[d - 1 - q % d] += (t % s) * w
        t //= s
        w *= s
    return tp


def head_sets(Hidx, s, d):
    sets = [0] * s
    for j in range(d - 1, -1, -1):
        sets[Hidx % s] |= 1 << j
        Hidx //= s
    return sets


def sum_range_addresses(tp, z, S, s, d, n_tail, m0, m1):
    pw = [s ** k for k in range(d + 1)]
    base, w = 0, []
    for j in range(d - 1, -1, -1):
        if (S >> j) & 1:
            base += z * n_tail * pw[d - 1 - j] + tp[j]
        else:
            base += pw[d] * tp[j]
            w.append(pw[d - 1 - j])
    n = len(w)
    c, off, m = [0] * n, 0, m0
    for i in range(n):
        c[i] = m % s
        m //= s
        off += c[i] * w[i]
    out = []
    for _ in range(m0, m1):
        out.append(base + off)
        for i in range(n):
            c[i] += 1
            if c[i] < s:
                off += w[i]
                break
            c[i] = 0
            off -= (s - 1) * w[i]
    return out


K_RT_CTA_TERMS, K_BLOCK = 2048, 256


def thread_or_warp_addresses(tp, z, S, s, d, n_tail):
    """A table entry's terms: one thread below 32 terms, 32 lanes with
    contiguous chunks below 2048, and from 2048 on the CTA's 256 threads with
    contiguous chunks, each a whole number of runs of the lowest digit
    (rt_fill_table, rt_chunk); without the table (sigma 2^d > 6000) one
    thread takes the whole range (rt_sum)."""
    terms = s ** (d - bin(S).count("1"))
    if terms < 32 or s << d > K_RT_TABLE:
        return sum_range_addresses(tp, z, S, s, d, n_tail, 0, terms)
    parts = 32 if terms < K_RT_CTA_TERMS else K_BLOCK
    per = (terms + parts - 1) // parts
    if s <= 8:
        per = (per + s - 1) // s * s  # whole runs of the lowest digit (rt_chunk)
    out = []
    for lane in range(parts):
        m0 = min(terms, lane * per)
        out += sum_range_addresses(tp, z, S, s, d, n_tail, m0, min(terms, m0 + per))
    return out


def deposit(v, mask):
    out, i = 0, 0
    while mask:
        b = mask & -mask
        if (v >> i) & 1:
            out |= b
        mask ^= b
        i += 1
    return out


def warp2_addresses(tp, z, S, d, n_tail):
    """sigma = 2, d >= 9: rt2_warp_sum's lanes and submask walk."""
    pw = [2 ** k for k in range(d + 1)]
    full = (1 << d) - 1
    base = sum(z * n_tail * pw[d - 1 - j] + tp[j] if (S >> j) & 1 else pw[d] * tp[j] for j in range(d))
    N = full ^ S
    bits = sum(1 << (d - 1 - j) for j in range(d) if (N >> j) & 1)  # bit reversal within d bits
    low, rest = 0, bits
    for _ in range(5):
        if not rest:
            break
        b = rest & -rest
        low |= b
        rest ^= b
    out = []
    for lane in range(32):
        if lane >= 1 << bin(low).count("1"):
            continue
        lo, sub = deposit(lane, low), 0
        while True:
            out.append(base + sub + lo)
            sub = (sub - rest) & rest
            if not sub:
                break
    return out


def kernel_candidates(x, s, d, h, warp2):
    """(z, k, sorted term addresses) for every candidate of state x, as the kernel forms them."""
    n_tail = s ** (d * (h - 1))
    t, Hidx = x % n_tail, x // n_tail
    tp = tail_parts(t, s, d, h)
    full = (1 << d) - 1
    if warp2:
        ones = sum(1 << j for j in range(d) if (Hidx >> (d - 1 - j)) & 1)
        sets = [full ^ ones, ones]
    else:
        sets = head_sets(Hidx, s, d)
    out, equal = [], False
    for z in range(s):
        if sets[z] == full:
            equal = True
            continue
        k = d - bin(sets[z]).count("1")
        addr = warp2_addresses(tp, z, sets[z], d, n_tail) if warp2 else thread_or_warp_addresses(
            tp, z, sets[z], s, d, n_tail)
        out.append((z, k, sorted(addr)))
    return out, equal


def check_states(s, d, h, xs):
    warp2 = s == 2 and d >= K_RT_WARP_D
    for x in xs:
        strings = decode(int(x), s, d, h)
        assert state_index(strings, s, h) == x
        got, equal = kernel_candidates(int(x), s, d, h, warp2)
        assert equal == all(st[0] == strings[0][0] for st in strings)
        want = [(z,) + defined_terms(strings, z, s)[::-1] for z in range(s)
                if not all(st[0] == z for st in strings)]
        assert [(z, k, a) for z, k, a in got] == [(z, k, a) for z, k, a in want], x


SMALL = [(2, 2, 3), (2, 3, 2), (2, 6, 2), (3, 2, 2), (3, 4, 1), (4, 3, 1), (5, 2, 2), (7, 2, 1), (10, 2, 1)]


@pytest.mark.parametrize("s,d,h", SMALL)
def test_every_state_every_candidate(s, d, h):
    assert rt_d_of(s ** (d * h), s, h) == d
    check_states(s, d, h, range(s ** (d * h)))


# (shape, random states besides the first, middle and last one); (3, 10, 1)
# has the largest sigma = 3 table (3072 entries, warp chunks of up to 3^10
# terms); (3, 11, 1), the first without a table, follows below
SAMPLED = [((2, 9, 2), 12), ((2, 12, 1), 12), ((2, 16, 1), 3), ((3, 6, 1), 12), ((3, 10, 1), 2), ((6, 3, 2), 12),
           ((9, 4, 1), 6), ((10, 4, 1), 4)]


@pytest.mark.parametrize("shape,n_random", SAMPLED, ids=lambda v: str(v))
def test_sampled_states(shape, n_random):
    s, d, h = shape
    n = s ** (d * h)
    assert rt_d_of(n, s, h) == d
    rng = np.random.default_rng(s * 100 + d * 10 + h)
    xs = [0, n // 2, n - 1] + [int(v) for v in rng.integers(0, n, n_random)]
    check_states(s, d, h, xs)


def test_one_state_without_the_table_at_d_11():
    """sigma = 3, d = 11 (no table): a state with heads of all three letters."""
    s, d, h = 3, 11, 1
    strings = [[j % 3] for j in range(d)]
    check_states(s, d, h, [state_index(strings, s, h)])


@pytest.mark.parametrize("s,d", [(2, 2), (2, 8), (3, 4), (3, 7), (5, 4), (7, 3), (10, 2), (10, 3)])
def test_table_entries(s, d):
    """Where the table fits (sigma 2^d <= 6000), fill writes every entry a
    lookup reads exactly once (threads below 32 terms, warps from 32 on), and
    distinct (z, S) take distinct entries; S = {} is one entry for every z."""
    full = (1 << d) - 1
    assert s << d <= K_RT_TABLE
    filled = []
    for e in range(s << d):
        z, S = e >> d, e & full
        if S == full or (S == 0 and z > 0):
            continue
        filled.append(e)
    read = set()
    for Hidx in range(s ** d):
        for z, S in enumerate(head_sets(Hidx, s, d)):
            if S != full:
                read.add((z << d) | S if S else 0)
    assert read <= set(filled)
    assert len(set(filled)) == len(filled)
