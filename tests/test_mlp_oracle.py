"""Pins of the warm-start network's CPU reference (oracle/mlp.py).

The analytic gradient is checked against central finite differences of the
loss (a computation that shares nothing with the backward formulas), and the
features against hand-worked examples and the orbit symmetry they must have.
"""
import numpy as np
import pytest

from oracle import mlp


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, scale, (mlp.HIDDEN, mlp.N_FEAT)),
        "b1": rng.normal(0, scale, mlp.HIDDEN),
        "W2": rng.normal(0, scale / 4, (mlp.HIDDEN, mlp.HIDDEN)),
        "b2": rng.normal(0, scale, mlp.HIDDEN),
        "w3": rng.normal(0, scale, mlp.HIDDEN),
        "b3": np.array(rng.normal(0, scale)),
    }


def test_features_hand_example():
    # h = 3, a = 101, b = 011: pairs (a_p, b_p) = (1,0), (0,1), (1,1) -> x = 0b10_01_11 = 39
    x = np.array([39])
    X = mlp.features(x, 3)[0]
    # canonical index: min over {39, 63-39=24, swap(39)=0b01_10_11=27, 63-27=36} = 24 = 0b01_10_00
    # -> a = 010, b = 100
    want = np.zeros(mlp.N_FEAT)
    for p, (a, b) in enumerate([(0, 1), (1, 0), (0, 0)]):
        want[4 * p + a] = 1
        want[4 * p + 2 + b] = 1
    want[-1] = 3 / 16
    assert np.array_equal(X, want)


@pytest.mark.parametrize("h", [2, 5, 13])
def test_features_invariant_under_orbit(h):
    rng = np.random.default_rng(h)
    x = rng.integers(0, 1 << (2 * h), size=200)
    n = 1 << (2 * h)
    swap = ((x >> 1) & 0x5555555555555555) | ((x & 0x5555555555555555) << 1)
    F = mlp.features(x, h)
    for y in (n - 1 - x, swap, n - 1 - swap):
        assert np.array_equal(mlp.features(y, h), F)
    assert np.all(F[:, 4 * min(h, mlp.H_IN):-1] == 0)


def test_gradient_matches_finite_differences():
    P = _params(3)
    rng = np.random.default_rng(4)
    hs = [4, 7, 12]
    X = np.concatenate([mlp.features(rng.integers(0, 1 << (2 * h), 6), h) for h in hs])
    t = rng.normal(0, 1, X.shape[0])
    loss, g = mlp.loss_and_grads(P, X, t)
    eps = 1e-6
    for name in P:
        flat = P[name].reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + eps
            lp, _ = mlp.loss_and_grads(P, X, t)
            flat[i] = old - eps
            lm, _ = mlp.loss_and_grads(P, X, t)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[i]) <= 1e-6 + 1e-5 * abs(fd), (name, i)


def test_gelu_is_the_erf_form():
    z = np.linspace(-4, 4, 17)
    from math import erf, sqrt

    assert np.allclose(mlp.gelu(z), [0.5 * v * (1 + erf(v / sqrt(2))) for v in z], atol=1e-15)


def test_bf16_rounding_is_nearest_even():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 in [1, 2)
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -9, -2.5 - 2.0 ** -7, 0.0])
    want = np.array([1.0, 1.0, 1 + 2 * 2.0 ** -7, 1.0, -2.5, 0.0])
    # the two ties (1 + 2^-8 and 1 + 3 2^-8) go to the neighbour with an even last bit
    assert np.array_equal(mlp.to_bf16(vals), want)
    got = mlp.to_bf16(np.random.default_rng(0).normal(0, 100, 1000))
    # every result is representable: the low 16 bits of its float32 are zero
    assert np.all(got.astype(np.float32).view(np.uint32) & 0xFFFF == 0)


def test_bf16_forward_differs_by_rounding_only():
    P = _params(3)
    X = mlp.features(np.random.default_rng(3).integers(0, 1 << 20, size=500), 10)
    y, _ = mlp.forward(P, X)
    yb = mlp.forward_bf16(P, X)
    diff = np.max(np.abs(y - yb))
    assert 0 < diff <= 1e-2 * np.max(np.abs(y))
    # a first layer whose GELU output is representable (GELU(40) = 40) and
    # parameters already in bfloat16: the rounded network is the network
    P2 = {k: mlp.to_bf16(v) for k, v in P.items()}
    P2["W1"] = np.zeros_like(P2["W1"])
    P2["b1"] = np.full(mlp.HIDDEN, 40.0)
    y2, _ = mlp.forward(P2, X)
    assert np.array_equal(mlp.forward_bf16(P2, X), y2)
