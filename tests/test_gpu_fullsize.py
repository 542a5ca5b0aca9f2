"""GPU parity at the benchmark's full size: sigma = d = 2, h = 16 (2^32 states).

The oracle cannot hold 32 GiB vectors, so the arguments of F are defined by a
counter-based generator that both sides implement from its published
definition (SplitMix64; torch on the GPU here, C in the oracle):
    v_k[y] = base_k + (SplitMix64(seed_k, c(y)) mod 2^46)
with c(y) = y, or c(y) = min(y, N-1-y) for complement-symmetric inputs.  The
CUDA sweep runs over every state; the oracle evaluates F at sampled states
(the first and last tiles plus random ones) and the two must agree bit for
bit.  The last test runs the benchmark's configuration to its published bound.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

S, D, H = 2, 2, 16
N = S ** (D * H)
K = 44
SPREAD_BITS = 46
SEEDS = [0x51ED2701, 0x0BADC0DE]
BASES = [(300 << K), (299 << K) + (1 << 40)]
GOLD = 0x9E3779B97F4A7C15


def _as_i64(c):
    return c - (1 << 64) if c >= 1 << 63 else c


@pytest.fixture(scope="module")
def torch_mod():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if free < 120 * 2 ** 30:
        pytest.skip("needs about 120 GiB of free device memory")
    return torch


def splitmix_fill(torch, out, seed, base, start, symmetric, chunk=1 << 28):
    """out[i] = base + (SplitMix64(seed, c(start + i)) mod 2^SPREAD_BITS), in int64 with wrap-around.

    c(y) = y (symmetric 0), min(y, N-1-y) (1), or the smallest index of y's
    orbit under complement and string swap (2).
    """
    g = _as_i64(GOLD)
    m1, m2 = _as_i64(0xBF58476D1CE4E5B9), _as_i64(0x94D049BB133111EB)
    ev = 0x5555555555555555
    n = out.numel()
    for off in range(0, n, chunk):
        m = min(chunk, n - off)
        y = torch.arange(start + off, start + off + m, dtype=torch.int64, device=out.device)
        if symmetric:
            c = torch.minimum(y, (N - 1) - y)
            if symmetric == 2:
                w = ((y >> 1) & ev) | ((y & ev) << 1)
                c = torch.minimum(c, torch.minimum(w, (N - 1) - w))
            y = c
        z = (y + 1) * g + seed
        z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * m1
        z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * m2
        z = z ^ ((z >> 31) & ((1 << 33) - 1))
        out[off:off + m] = base + (z & ((1 << SPREAD_BITS) - 1))


def sample_states(rng, count=3000):
    edges = np.concatenate([np.arange(0, 2048), np.arange(N - 2048, N),
                            np.arange(N // 4 - 1024, N // 4 + 1024), np.arange(N // 2 - 1024, N // 2 + 1024)])
    rnd = rng.integers(0, N, size=count, dtype=np.int64)
    return np.unique(np.concatenate([edges, rnd])).astype(np.int64)


def test_generator_matches_oracle(torch_mod, orc):
    torch = torch_mod
    out = torch.empty(64, dtype=torch.int64, device="cuda")
    splitmix_fill(torch, out, SEEDS[0], 0, 12345, False)
    got = out.cpu().numpy()
    want = [orc.splitmix64_at(SEEDS[0], 12345 + i) % (1 << SPREAD_BITS) for i in range(64)]
    assert list(got) == want


def test_h16_stateless_sweep_sampled(torch_mod, orc):
    import paper_2407_10925_gb300 as lb

    torch = torch_mod
    v1 = torch.empty(N, dtype=torch.int64, device="cuda")
    v2 = torch.empty(N, dtype=torch.int64, device="cuda")
    splitmix_fill(torch, v1, SEEDS[0], BASES[0], 0, False)
    splitmix_fill(torch, v2, SEEDS[1], BASES[1], 0, False)
    torch.cuda.synchronize()
    out = torch.empty(N, dtype=torch.int64, device="cuda")
    lb.lcs_sweep_fx(S, D, H, [v1, v2], out)
    torch.cuda.synchronize()
    xs = sample_states(np.random.default_rng(2024))
    got = out[torch.from_numpy(xs).cuda()].cpu().numpy()
    want = orc.F_generated(S, D, H, SEEDS, BASES, 1 << SPREAD_BITS, xs.astype(np.uint64))
    del v1, v2, out
    torch.cuda.empty_cache()
    assert np.array_equal(got, want), xs[got != want][:10]


@pytest.mark.parametrize("symmetric", [1, 2], ids=["complement", "complement+swap"])
def test_h16_symmetric_iteration_sampled(torch_mod, orc, symmetric):
    """The library's symmetric sweeps with the fused increment reduction, at full size.

    Complement-symmetric arguments run the complement kernel; arguments that are
    also swap-symmetric run the kernel that uses both symmetries (the one the
    benchmark's zero start runs).
    """
    import paper_2407_10925_gb300 as lb

    torch = torch_mod
    newest = torch.empty(N, dtype=torch.int64, device="cuda")
    older = torch.empty(N, dtype=torch.int64, device="cuda")
    splitmix_fill(torch, newest, SEEDS[0], BASES[0], 0, symmetric)
    splitmix_fill(torch, older, SEEDS[1], BASES[1], 0, symmetric)
    torch.cuda.synchronize()  # the library reads them on its own stream
    with lb.LcsBound(S, D, H, symmetry=1) as hnd:
        hnd.set_start_fx([newest, older])
        del newest, older
        torch.cuda.empty_cache()
        hnd.iterate(1)
        rep = hnd.report()
        out = torch.empty(N, dtype=torch.int64, device="cuda")
        lb.lcs_bound_export_fx(hnd.hnd, 0, out)
        torch.cuda.synchronize()
    xs = sample_states(np.random.default_rng(7))
    xs = np.unique(np.concatenate([xs, [rep["argmin"]]]))
    got = out[torch.from_numpy(xs).cuda()].cpu().numpy()
    del out
    torch.cuda.empty_cache()
    # the oracle reads the same symmetric generator
    canon = np.minimum(xs, N - 1 - xs)
    if symmetric == 2:
        w = ((xs >> 1) & 0x5555555555555555) | ((xs & 0x5555555555555555) << 1)
        canon = np.minimum(canon, np.minimum(w, N - 1 - w))
    want = orc.F_generated(S, D, H, SEEDS, BASES, 1 << SPREAD_BITS, xs.astype(np.uint64), symmetric=symmetric)
    assert np.array_equal(got, want)
    # R is attained at its state, and no sampled state has a smaller increment
    prev = np.array([BASES[0] + orc.splitmix64_at(SEEDS[0], int(c)) % (1 << SPREAD_BITS) for c in canon])
    inc = got - prev
    i = int(np.flatnonzero(xs == rep["argmin"])[0])
    assert inc[i] == rep["R"]
    assert inc.min() >= rep["R"]


def test_h16_bound_matches_table2(torch_mod):
    """The benchmark's configuration (2^32 states, zero start, 2000 iterations): Table 2's 0.789021."""
    import paper_2407_10925_gb300 as lb

    with lb.LcsBound(S, D, H, check_every=100) as hnd:
        hnd.iterate(2000)
        bound, argmin, r, eps, at_iter = hnd.read()
    assert math.floor(bound * 1e6 + 1e-9) / 1e6 == pytest.approx(0.789021, abs=1e-9)
    assert bound < 0.826280
