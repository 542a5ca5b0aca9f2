"""GPU parity of the general kernels (shapes without a specialised kernel: d up
to 16, sigma up to 10, full storage, the paper's F) against the CPU oracle,
bit for bit: the stateless sweep on random arguments, whole runs of Algorithm
2 (iterates, R and its state, E, the kept triplet, the bound) from the zero
start and from random starts, and the feasibility check of a given vector.

The shapes cover every way the kernels form candidates.  Handles with h >= 2
and sigma^d <= 16384 run the block form (a means table filled from blocks of
sigma^d consecutive values staged in shared memory, then one thread per
state).  The stateless sweep and h = 1 run the one-pass kernels: the shared
table of sums (sigma * 2^d <= 6000 entries) filled by one CTA per tail tuple,
or by one warp per tuple for small tables and many tuples, and, for sigma = 2
from d = 9 on, one warp per state.  At the benchmark shapes (3, 8, 2) and
(2, 12, 2) the oracle's plain F (2631 and 259 terms per state) is too slow for
every state, so windows of states are compared, and the increment reduction
against the exported iterate.  A small number of fractional bits keeps the sums of
sigma^d terms inside int64 (the library checks that headroom for its handles).
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

K = 30

# (6, 2, 4) and (10, 2, 3) have small tables and at least 8192 tail tuples:
# one warp per tuple instead of one CTA
SWEEP_SHAPES = [(2, 6, 2), (2, 7, 1), (2, 9, 2), (2, 10, 1), (2, 12, 1), (2, 13, 1), (3, 4, 2), (3, 5, 1),
                (4, 3, 2), (5, 3, 1), (6, 2, 2), (7, 3, 1), (8, 2, 3), (10, 2, 2), (9, 4, 1), (6, 2, 4), (10, 2, 3)]


@pytest.fixture(scope="module")
def lb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return lb


@pytest.mark.parametrize("s,d,h", SWEEP_SHAPES)
def test_general_stateless_sweep_bit_exact(lb, orc, s, d, h):
    import torch

    vs = inputs.random_history(s, d, h, seed=300 + 11 * s + 3 * d + h, frac_bits=K)
    want = orc.F(s, d, h, vs, arith="fx", frac_bits=K)
    dev = [torch.from_numpy(v).cuda() for v in vs]
    out = torch.empty(want.size, dtype=torch.int64, device="cuda")
    lb.lcs_sweep_fx(s, d, h, dev, out, frac_bits=K)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]


RUN_CASES = [
    # s, d, h, iters, check_every, r_mode, random start
    (2, 6, 2, 20, 5, 0, False),
    (2, 12, 1, 12, 0, 0, False),
    (2, 9, 2, 10, 5, 0, True),
    (2, 7, 1, 25, 3, 1, True),
    (3, 4, 2, 15, 3, 0, False),
    (3, 5, 1, 20, 4, 0, True),
    (4, 3, 2, 12, 4, 0, False),
    (6, 2, 2, 20, 5, 1, False),
    (10, 2, 3, 12, 4, 0, True),
    (10, 2, 2, 12, 0, 0, True),
    (5, 3, 1, 20, 1, 0, False),
    # the block form (h >= 2): one block per tile, several (sigma^d < 2048)
    # with a partial last tile, sigma = 2 with large d
    (2, 10, 2, 2, 1, 0, True),
    (3, 6, 2, 3, 2, 1, True),
    (2, 8, 2, 5, 5, 0, True),
    (6, 2, 3, 6, 3, 0, True),
    (7, 2, 2, 5, 5, 1, True),
    (4, 4, 2, 4, 2, 0, True),
    (5, 3, 2, 6, 3, 0, True),
    (9, 3, 2, 2, 1, 0, True),
    (2, 6, 3, 4, 2, 0, True),
]


@pytest.mark.parametrize("case", RUN_CASES, ids=lambda c: "s%d_d%d_h%d_it%d_ce%d_r%d_rand%d" % c)
def test_general_run_bit_exact(lb, orc, case):
    s, d, h, iters, check_every, r_mode, rand = case
    start = None
    if rand:
        hist = inputs.random_history(s, d, h, seed=900 + s + d + h, frac_bits=K)
        start = [hist[d - 1 - k] for k in range(d)]  # oldest first
    want = orc.run(s, d, h, iters, arith="fx", check_every=check_every, r_mode=r_mode, frac_bits=K, start=start)
    with lb.LcsBound(s, d, h, check_every=check_every, r_mode=r_mode, frac_bits=K) as hnd:
        assert hnd.n_stored == hnd.n_states  # full storage
        if start is not None:
            hnd.set_start_fx([start[d - 1 - k] for k in range(d)])
        hnd.iterate(iters)
        rep = hnd.report()
        for k in range(d):
            got = hnd.export_fx(k)
            assert np.array_equal(got, want["iterates"][k]), (k, np.flatnonzero(got != want["iterates"][k])[:10])
        assert (rep["R"], rep["argmin"], rep["E"]) == (want["R"], want["argmin"], want["E"])
        assert (rep["r"], rep["eps"], rep["kept_iter"]) == (want["r"], want["eps"], want["kept_iter"])
        assert rep["status"] == 0
        assert hnd.read()[0] == want["bound_rd"]


@pytest.mark.parametrize("s,d,h", [(3, 4, 2), (2, 12, 1), (2, 9, 2), (10, 2, 2), (7, 3, 1), (6, 2, 3), (2, 10, 2)])
def test_general_check_vector_matches_oracle(lb, orc, s, d, h):
    import torch

    u = inputs.random_fx(s, d, h, seed=77 + s + d + h, frac_bits=K)
    one = 1 << K
    for R in [int(0.3 * one), int(0.45 * one), -(1 << 20)]:
        E_want, _ = orc.check(s, d, h, u, R, arith="fx", frac_bits=K)
        with lb.LcsBound(s, d, h, frac_bits=K) as hnd:
            E_got = hnd.check_vector(torch.from_numpy(u).cuda(), R)
        assert E_got == E_want, R


def test_general_kernel_is_counted(lb):
    with lb.LcsBound(3, 4, 2, timing=1, frac_bits=K) as hnd:
        hnd.iterate(3)
        assert hnd.stats()["sweep_bytes"] == 3 * 8 * (4 + 1) * 3 ** 8


def test_all_advance_sets_stay_unsupported_without_a_kernel(lb):
    with pytest.raises(lb.LcsError) as e:
        lb.LcsBound(3, 4, 2, f_mode=1)
    assert e.value.status == lb.LCS_EUNSUPPORTED


@pytest.mark.parametrize("s,d,h", [(3, 8, 2), (2, 12, 2)])
def test_block_form_sampled_at_benchmark_shapes(lb, orc, s, d, h):
    kb = 36  # the benchmark's fractional bits for these shapes
    hist = inputs.random_history(s, d, h, seed=4242 + s + d, frac_bits=kb)  # newest first
    n = hist[0].size
    with lb.LcsBound(s, d, h, check_every=1, frac_bits=kb) as hnd:
        hnd.set_start_fx(hist)
        hnd.iterate(1)
        rep = hnd.report()
        got = hnd.export_fx(0)
    assert rep["status"] == 0
    rng = np.random.default_rng(17)
    sd = s ** d
    # windows: the first and last states, and random ones across head and tail digits
    starts = [0, n - 2 * sd] + [int(x) for x in rng.integers(0, n - 2 * sd, size=4)]
    for x0 in starts:
        want = orc.F(s, d, h, hist, arith="fx", frac_bits=kb, x0=x0, x1=x0 + 2 * sd)
        part = got[x0:x0 + 2 * sd]
        assert np.array_equal(part, want), (x0, np.flatnonzero(part != want)[:10])
    inc = got - hist[0]
    assert rep["R"] == int(inc.min())
    assert inc[rep["argmin"]] == rep["R"]
