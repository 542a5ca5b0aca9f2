"""The oracle's F on generated arguments (used by the full-size GPU parity tests,
whose vectors the oracle cannot hold) against its plain F on the same
arguments written out.

The arguments are v_k[y] = base_k + (SplitMix64(seed_k, c(y)) mod spread),
with c(y) a canonical member of y's orbit under the symmetries asked for.
Here c is restated with plain Python digit arithmetic from the state index
(string j's letter at position p has weight sigma^(d (h-1-p) + (d-1-j))),
the vectors are built explicitly at small sizes, and the two oracle entry
points must agree at every state.  The vectors must also have the symmetry
the mode promises.
"""
import itertools

import numpy as np
import pytest

SEEDS = [0x51ED2701, 0x0BADC0DE, 0x1234567]
BASES = [(300 << 44), (299 << 44) + (1 << 40), (298 << 44) + (3 << 40)]
SPREAD = 1 << 46


def _digits(s, d, h, y):
    """digits[p][j]: string j's letter at position p (0 = head)."""
    out = [[0] * d for _ in range(h)]
    for p in range(h):
        for j in range(d):
            out[p][j] = (y // s ** (d * (h - 1 - p) + (d - 1 - j))) % s
    return out


def _index(s, d, h, digits):
    return sum(digits[p][j] * s ** (d * (h - 1 - p) + (d - 1 - j)) for p in range(h) for j in range(d))


def _images(s, d, h, y, symmetric):
    """y's images under the symmetries of the mode (y itself included)."""
    X = _digits(s, d, h, y)
    orders = [tuple(range(d))]
    if symmetric == 2 or symmetric == 3:
        orders = list(itertools.permutations(range(d)))
    out = []
    for order in orders:
        Y = [[X[p][order[j]] for j in range(d)] for p in range(h)]
        out.append(_index(s, d, h, Y))
        if symmetric:
            out.append(_index(s, d, h, [[s - 1 - Y[p][j] for j in range(d)] for p in range(h)]))
    return out


def _explicit(orc, s, d, h, symmetric):
    n = s ** (d * h)
    canon = [min(_images(s, d, h, y, symmetric)) for y in range(n)]
    return [np.array([BASES[k] + orc.splitmix64_at(SEEDS[k], c) % SPREAD for c in canon], dtype=np.int64)
            for k in range(d)], canon


@pytest.mark.parametrize("s,d,h,symmetric", [(2, 2, 4, 0), (2, 2, 4, 1), (2, 2, 4, 2), (3, 2, 2, 0),
                                             (2, 3, 3, 0), (2, 3, 3, 1), (2, 3, 3, 3)])
def test_generated_arguments_match_plain_F(orc, s, d, h, symmetric):
    vs, canon = _explicit(orc, s, d, h, symmetric)
    n = s ** (d * h)
    xs = np.arange(n, dtype=np.uint64)
    want = orc.F(s, d, h, vs, arith="fx")
    got = orc.F_generated(s, d, h, SEEDS[:d], BASES[:d], SPREAD, xs, symmetric=symmetric)
    assert np.array_equal(got, want)
    # the promised symmetry holds for the arguments
    for y in range(n):
        for w in _images(s, d, h, y, symmetric):
            assert canon[w] == canon[y]


def test_generated_symmetric_modes_need_their_shapes(orc):
    xs = np.arange(4, dtype=np.uint64)
    with pytest.raises(Exception):
        orc.F_generated(2, 2, 3, SEEDS[:2], BASES[:2], SPREAD, xs, symmetric=3)
    with pytest.raises(Exception):
        orc.F_generated(2, 3, 2, SEEDS[:3], BASES[:3], SPREAD, xs, symmetric=2)
    with pytest.raises(Exception):
        orc.F_generated(3, 2, 2, SEEDS[:2], BASES[:2], SPREAD, xs, symmetric=1)


def test_splitmix64_matches_its_published_outputs(orc):
    """The generator both sides implement from its definition, against the
    first outputs of the published SplitMix64 from state 0."""
    from conftest import load_golden

    rows = load_golden("splitmix64_seed0.txt")
    assert len(rows) >= 4
    for seed, i, out in rows:
        assert orc.splitmix64_at(int(seed), int(i)) == int(out, 16)


def test_gpu_side_generators_match_the_published_outputs():
    """The torch restatements the full-size GPU tests fill their vectors with,
    run on CPU tensors, give the published outputs' low 46 bits (the spread
    those tests take)."""
    import torch

    from conftest import load_golden
    import test_gpu_d3_fullsize as g3
    import test_gpu_fullsize as g2

    rows = [(int(s), int(i), int(o, 16)) for s, i, o in load_golden("splitmix64_seed0.txt")]
    assert {s for s, _, _ in rows} == {0}
    want = [o & ((1 << g2.SPREAD_BITS) - 1) for _, _, o in rows]
    out = torch.empty(len(rows), dtype=torch.int64)
    g2.splitmix_fill(torch, out, 0, 0, 0, 0)
    assert out.tolist() == want
    assert g3.SPREAD_BITS == g2.SPREAD_BITS
    assert g3.splitmix(torch, torch.arange(len(rows), dtype=torch.int64), 0, 0).tolist() == want


def test_gpu_side_canonical_maps_match_the_orbits(orc):
    """The full-size GPU tests' canonical members, on CPU tensors at their own
    sizes (sampled states), against the orbits enumerated with plain digit
    arithmetic: sigma = 2, d = 3, h = 11 under the string orders and the
    complement; sigma = d = 2, h = 16 under the swap and the complement
    (through the generated values, which read the canonical member)."""
    import torch

    import test_gpu_d3_fullsize as g3
    import test_gpu_fullsize as g2

    rng = np.random.default_rng(2407)
    ys = [0, 1, 2, 7, g3.N // 2 - 1, g3.N // 2, g3.N - 1] + [int(v) for v in rng.integers(0, g3.N, 300)]
    got = g3.canonical(torch, torch.tensor(ys, dtype=torch.int64)).tolist()
    assert got == [min(_images(2, 3, g3.H, y, 3)) for y in ys]

    mask = (1 << g2.SPREAD_BITS) - 1
    ys = [0, 5, g2.N // 2, g2.N - 1] + [int(v) for v in rng.integers(0, g2.N, 100)]
    for y in ys:
        out = torch.empty(1, dtype=torch.int64)
        g2.splitmix_fill(torch, out, g2.SEEDS[0], 0, y, 2)
        c = min(_images(2, 2, g2.H, y, 2))
        assert out.item() == orc.splitmix64_at(g2.SEEDS[0], c) & mask, y
