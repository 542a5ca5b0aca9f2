"""The orbit form's layout as include/lcs_bound.h defines it (sigma = d = 2),
checked from the definition alone, with plain index arithmetic:

* the representatives (s, a, beta), 0 <= a <= beta < K = 2^(h-2), take the
  places q = s K (K + 1) / 2 + beta (beta + 1) / 2 + a, every place in
  [0, K (K + 1)) once, so the form has 4 K (K + 1) = 4^(h-1) + 2^h values;
* the eight stored states of the representatives' orbits (heads 00 and 01 of
  t = (a, b), ~t, t' = (~b, ~a), ~t' = (b, a)) cover every stored state
  (first string's head 0) and no other;
* on a vector with the complement and the swap symmetry, each orbit holds the
  four values the header lists: v(00, t) = v(00, ~t'), v(00, ~t) = v(00, t'),
  v(01, t) = v(01, t'), v(01, ~t) = v(01, ~t').
"""
import numpy as np
import pytest


def index(h, g0, g1, a, b):
    """STATE INDEX of strings g0 a and g1 b (a, b: (h-1)-bit integers, most significant letter first)."""
    x = (g0 << (2 * h - 1)) | (g1 << (2 * h - 2))
    for i in range(h - 1):
        x |= ((a >> i) & 1) << (2 * i + 1) | ((b >> i) & 1) << (2 * i)
    return x


def representatives(h):
    K, M = 1 << (h - 2), (1 << (h - 1)) - 1
    for s in (0, 1):
        for beta in range(K):
            for a in range(beta + 1):
                b = beta if s == 0 else M - beta
                yield s * (K * (K + 1) // 2) + beta * (beta + 1) // 2 + a, a, b


@pytest.mark.parametrize("h", [2, 3, 4, 5, 6, 7])
def test_places_and_coverage(h):
    K, M = 1 << (h - 2), (1 << (h - 1)) - 1
    places, covered = [], set()
    for q, a, b in representatives(h):
        places.append(q)
        for g1 in (0, 1):
            for ta, tb in [(a, b), (M - a, M - b), (M - b, M - a), (b, a)]:
                covered.add(index(h, 0, g1, ta, tb))
    assert sorted(places) == list(range(K * (K + 1)))
    assert 4 * K * (K + 1) == 4 ** (h - 1) + 2 ** h
    assert covered == set(range(2 ** (2 * h - 1)))  # exactly the stored half


def symmetric_vector(h, seed):
    """A random vector invariant under the complement and the string swap."""
    n = 4 ** h
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 1 << 40, size=n, dtype=np.int64)
    x = np.arange(n, dtype=np.int64)
    w = ((x >> 1) & 0x5555555555555555) | ((x & 0x5555555555555555) << 1)
    images = [x, (n - 1) - x, w, (n - 1) - w]
    canon = np.minimum.reduce(images)
    return v[canon]


@pytest.mark.parametrize("h", [3, 5, 6])
def test_four_values_per_orbit(h):
    v = symmetric_vector(h, seed=h)
    M = (1 << (h - 1)) - 1
    for q, a, b in representatives(h):
        t, tc, tp, sw = (a, b), (M - a, M - b), (M - b, M - a), (b, a)
        assert v[index(h, 0, 0, *t)] == v[index(h, 0, 0, *sw)]
        assert v[index(h, 0, 0, *tc)] == v[index(h, 0, 0, *tp)]
        assert v[index(h, 0, 1, *t)] == v[index(h, 0, 1, *tp)]
        assert v[index(h, 0, 1, *tc)] == v[index(h, 0, 1, *sw)]
