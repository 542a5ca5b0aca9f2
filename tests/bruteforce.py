"""Brute-force W_n from its definition (paper section 2.1), for pinning the oracle.

W_n(a_1..a_d) = E[ max_{i_1+..+i_d = n} L(a_1 x_1[..i_1], .., a_d x_d[..i_d]) ]
with x_j independent uniform random strings and L the length of a longest
common subsequence.  Everything here is computed exactly: the expectation is
an average over every outcome of the random characters (as a Fraction), and L
is the textbook LCS dynamic program over d strings.  Nothing in this module
uses the oracle or the feasible-triplet recursion.

The state index is the paper's interleaved index (section 3.2): digit of
string j at position p has weight sigma^(d (h-1-p) + (d-1-j)).
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def state_strings(sigma: int, d: int, h: int, x: int):
    """The d strings (head first) of the state with interleaved index x."""
    digits = []
    for _ in range(d * h):
        digits.append(x % sigma)
        x //= sigma
    digits.reverse()  # most significant first: position 0 string 0, position 0 string 1, ...
    return [tuple(digits[p * d + j] for p in range(h)) for j in range(d)]


def lcs_prefix_table(strings):
    """L[i_1,..,i_d] = LCS length of the prefixes of the given lengths (d-dimensional DP)."""
    d = len(strings)
    shape = tuple(len(s) + 1 for s in strings)
    L = np.zeros(shape, dtype=np.int64)
    for idx in itertools.product(*[range(1, m) for m in shape]):
        chars = [strings[j][idx[j] - 1] for j in range(d)]
        if all(c == chars[0] for c in chars):
            L[idx] = L[tuple(i - 1 for i in idx)] + 1
        else:
            best = 0
            for j in range(d):
                prev = list(idx)
                prev[j] -= 1
                v = L[tuple(prev)]
                if v > best:
                    best = v
            L[idx] = best
    return L


def compositions(n: int, d: int):
    """All (i_1..i_d) of non-negative integers with sum n."""
    if d == 1:
        yield (n,)
        return
    for i in range(n + 1):
        for rest in compositions(n - i, d - 1):
            yield (i,) + rest


def W_table(sigma: int, d: int, h: int, n_max: int):
    """W[n][x] for n = 0..n_max and every state x, as Fractions.

    One enumeration of all sigma^(d n_max) outcomes of the random suffixes
    serves every n <= n_max, because the first i_j characters of a uniform
    string of length n_max are themselves uniform.
    """
    N = sigma ** (d * h)
    totals = [[0] * N for _ in range(n_max + 1)]
    comps = [list(compositions(n, d)) for n in range(n_max + 1)]
    suffixes = list(itertools.product(range(sigma), repeat=n_max))
    count = 0
    for xs in itertools.product(suffixes, repeat=d):
        count += 1
        for x in range(N):
            a = state_strings(sigma, d, h, x)
            L = lcs_prefix_table([a[j] + xs[j] for j in range(d)])
            for n in range(n_max + 1):
                best = 0
                for comp in comps[n]:
                    v = L[tuple(h + i for i in comp)]
                    if v > best:
                        best = v
                totals[n][x] += int(best)
    return [[Fraction(t, count) for t in row] for row in totals]
