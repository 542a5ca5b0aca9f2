"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds no arithmetic of the method: it only draws vectors.  The
method itself starts from the zero vector (Algorithm 2), so the random
vectors here serve as arbitrary arguments of F and of the check, and as warm
starts.  Values are fixed-point integers (units of 2^-K) of the magnitude the
iterates reach (a few hundred units), spread over a few units like converged
iterates, plus a random component that exercises every index.
"""
from __future__ import annotations

import numpy as np

K_DEFAULT = 44


def n_states(sigma: int, d: int, h: int) -> int:
    return sigma ** (d * h)


def complement_index(n: int) -> np.ndarray:
    """N-1-x for every x (the complement map of sigma = 2, paper section 3.3)."""
    return np.arange(n - 1, -1, -1, dtype=np.int64)


def swap_index(n: int) -> np.ndarray:
    """The index with the two strings exchanged (sigma = d = 2, interleaved bits)."""
    y = np.arange(n, dtype=np.int64)
    return ((y >> 1) & 0x5555555555555555) | ((y & 0x5555555555555555) << 1)


def swap_index_d2(sigma: int, h: int) -> np.ndarray:
    """d = 2, any sigma: the index with the two strings exchanged (the two base-sigma
    digits of every position swapped in the interleaved index)."""
    n = sigma ** (2 * h)
    x = np.arange(n, dtype=np.int64)
    y = np.zeros(n, dtype=np.int64)
    m = 1
    for _ in range(h):
        pd = x % (sigma * sigma)
        x //= sigma * sigma
        y += ((pd % sigma) * sigma + pd // sigma) * m
        m *= sigma * sigma
    return y


def symmetrize(v: np.ndarray, swap: bool = False) -> np.ndarray:
    """The smallest value over each orbit of the complement map (and of the string swap)."""
    n = v.size
    out = np.minimum(v, v[complement_index(n)])
    if swap:
        out = np.minimum(out, out[swap_index(n)])
    return out


def perm_index_d3(h: int, perm) -> np.ndarray:
    """sigma = 2, d = 3: the index with string j moved to position perm[j]."""
    n = 8 ** h
    x = np.arange(n, dtype=np.int64)
    y = np.zeros(n, dtype=np.int64)
    for j in range(3):
        for i in range(h):
            y |= ((x >> (3 * i + 2 - j)) & 1) << (3 * i + 2 - perm[j])
    return y


def perm_symmetrize_d3(v: np.ndarray, h: int) -> np.ndarray:
    """sigma = 2, d = 3: the smallest value over each orbit of the string
    permutations and the complement (a vector with both symmetries)."""
    import itertools

    n = v.size
    out = v.copy()
    for perm in itertools.permutations(range(3)):
        y = perm_index_d3(h, perm)
        out = np.minimum(out, v[y])
        out = np.minimum(out, v[n - 1 - y])
    return out


def swap_symmetrize(v: np.ndarray, sigma: int, h: int) -> np.ndarray:
    """d = 2, any sigma: the smaller value of each pair of states exchanged by the string swap."""
    return np.minimum(v, v[swap_index_d2(sigma, h)])


def random_fx(sigma, d, h, seed, base_units=200.0, spread_units=4.0, frac_bits=K_DEFAULT, symmetric=False,
              swap=False):
    """One random fixed-point vector over all states."""
    rng = np.random.default_rng(seed)
    n = n_states(sigma, d, h)
    one = float(1 << frac_bits)
    v = (base_units + spread_units * rng.random(n)) * one
    v = v.astype(np.int64)
    v += rng.integers(0, 1 << 20, size=n, dtype=np.int64)  # low-order noise below the unit
    if sigma == 2 and d == 3 and swap:
        return perm_symmetrize_d3(v, h)
    if sigma != 2 and swap and not symmetric:
        if d != 2:
            raise ValueError("the swap needs d = 2")
        return swap_symmetrize(v, sigma, h)
    if symmetric or swap:
        if sigma != 2 or (swap and d != 2):
            raise ValueError("complement symmetry needs sigma = 2; the swap needs d = 2")
        v = symmetrize(v, swap)
    return v


def random_history(sigma, d, h, seed, step_units=0.4, frac_bits=K_DEFAULT, symmetric=False, swap=False):
    """d vectors shaped like consecutive iterates: v[k] is k steps older than v[0]."""
    base = random_fx(sigma, d, h, seed, frac_bits=frac_bits, symmetric=symmetric, swap=swap)
    one = 1 << frac_bits
    rng = np.random.default_rng(seed + 7919)
    n = base.size
    out = []
    for k in range(d):
        jitter = rng.integers(0, one // 16, size=n, dtype=np.int64)
        if sigma == 2 and d == 3 and swap:
            jitter = perm_symmetrize_d3(jitter, h)
        elif sigma != 2 and swap and not symmetric:
            jitter = swap_symmetrize(jitter, sigma, h)
        elif symmetric or swap:
            jitter = symmetrize(jitter, swap)
        out.append(base - int(k * step_units * one) - jitter)
    return out
