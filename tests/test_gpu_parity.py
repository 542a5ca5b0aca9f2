"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Fixed-point results are compared bit for bit (integer work): the iterates,
R and its state, E, the kept triplet and the bound.  Inputs are the paper's
zero start or seeded synthetic vectors (tests/inputs.py).
"""
import math

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

K = 44


@pytest.fixture(scope="module")
def lb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return lb


@pytest.fixture(scope="module")
def torch_mod():
    import torch

    return torch


SWEEP_SHAPES = [(2, 2, 1), (2, 2, 2), (2, 2, 3), (2, 2, 5), (2, 2, 7), (2, 3, 1), (2, 3, 2), (2, 3, 4),
                (2, 4, 1), (2, 4, 3), (2, 5, 2), (3, 2, 1), (3, 2, 2), (3, 2, 4), (3, 3, 2), (4, 2, 1),
                (4, 2, 3), (5, 2, 2)]


@pytest.mark.parametrize("s,d,h", SWEEP_SHAPES)
def test_stateless_sweep_bit_exact(lb, torch_mod, orc, s, d, h):
    """v_out = F(v_prev) on random arguments: every state, bit for bit."""
    torch = torch_mod
    vs = inputs.random_history(s, d, h, seed=100 + 7 * h + d + s)
    want = orc.F(s, d, h, vs, arith="fx")
    dev = [torch.from_numpy(v).cuda() for v in vs]
    out = torch.empty(want.size, dtype=torch.int64, device="cuda")
    lb.lcs_sweep_fx(s, d, h, dev, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, want), np.flatnonzero(got != want)[:10]


RUN_CASES = [
    # s, d, h, iters, check_every, symmetry, r_mode
    (2, 2, 1, 30, 0, 1, 0),
    (2, 2, 3, 57, 5, 1, 0),
    (2, 2, 5, 80, 0, 1, 0),
    (2, 2, 5, 33, 1, 0, 0),
    (2, 2, 6, 41, 7, 1, 1),
    (2, 3, 2, 45, 4, 1, 0),
    (2, 3, 3, 30, 0, 0, 0),
    (2, 4, 2, 25, 0, 1, 0),
    (2, 5, 1, 35, 3, 1, 0),
    (3, 2, 2, 40, 3, 1, 0),
    (3, 2, 3, 21, 0, 1, 0),
    (4, 2, 2, 22, 5, 1, 0),
    (5, 2, 1, 30, 0, 1, 0),
    (3, 3, 1, 25, 2, 1, 0),
]


def _check_run_against_oracle(lb, orc, s, d, h, iters, check_every, symmetry, r_mode, start=None, f_mode=0):
    want = orc.run(s, d, h, iters, arith="fx", check_every=check_every, r_mode=r_mode, start=start, f_mode=f_mode)
    with lb.LcsBound(s, d, h, check_every=check_every, symmetry=symmetry, r_mode=r_mode, f_mode=f_mode) as hnd:
        if start is not None:
            # start[k] is v_k (oldest first); the library takes newest first
            hnd.set_start_fx([start[d - 1 - k] for k in range(d)])
        hnd.iterate(iters)
        rep = hnd.report()
        for k in range(d):
            got = hnd.export_fx(k)
            assert np.array_equal(got, want["iterates"][k]), (k, np.flatnonzero(got != want["iterates"][k])[:10])
        assert rep["R"] == want["R"]
        assert rep["argmin"] == want["argmin"]
        assert rep["E"] == want["E"]
        assert (rep["r"], rep["eps"], rep["kept_iter"]) == (want["r"], want["eps"], want["kept_iter"])
        assert rep["status"] == 0
        bound, argmin, r, eps, at_iter = hnd.read()
        assert bound == want["bound_rd"]
        assert at_iter == want["kept_iter"]


@pytest.mark.parametrize("case", RUN_CASES, ids=lambda c: "s%d_d%d_h%d_it%d_ce%d_sym%d_r%d" % c)
def test_run_bit_exact(lb, orc, case):
    _check_run_against_oracle(lb, orc, *case)


@pytest.mark.parametrize("s,d,h,sym", [(2, 2, 4, 1), (2, 2, 4, 0), (2, 3, 2, 1), (3, 2, 2, 0)])
def test_warm_start_bit_exact(lb, orc, s, d, h, sym):
    hist = inputs.random_history(s, d, h, seed=5 + h, symmetric=(s == 2))
    start = [hist[d - 1 - k] for k in range(d)]  # oldest first
    _check_run_against_oracle(lb, orc, s, d, h, 17, 4, sym, 0, start=start)


@pytest.mark.parametrize("h", [6, 7, 9])
@pytest.mark.parametrize("swap", [False, True])
def test_sigma2_d2_paths_bit_exact(lb, orc, h, swap):
    """sigma = d = 2, h >= 6: swap-symmetric starts run the kernel that also uses the
    string swap; complement-only starts fall back to the complement kernel.  Both exact."""
    hist = inputs.random_history(2, 2, h, seed=40 + h, symmetric=True, swap=swap)
    start = [hist[1], hist[0]]  # oldest first
    _check_run_against_oracle(lb, orc, 2, 2, h, 23, 6, 1, 0, start=start)


@pytest.mark.parametrize("h", [6, 8, 11])
def test_swap_kernel_zero_start_many_checks(lb, orc, h):
    """Zero start (swap-symmetric): every iteration checked, r_mode both ways."""
    for r_mode in (0, 1):
        _check_run_against_oracle(lb, orc, 2, 2, h, 12 if h > 8 else 30, 1, 1, r_mode)


D2S_SHAPES = [(3, 4), (3, 5), (4, 3), (4, 4), (5, 3)]


@pytest.mark.parametrize("s,h", D2S_SHAPES)
@pytest.mark.parametrize("swap", [False, True])
def test_d2_swap_paths_bit_exact(lb, orc, s, h, swap):
    """d = 2, sigma >= 3: swap-symmetric starts run the kernels that read each
    value of v_{t-1} once through the string swap; other starts run the generic
    kernels.  Both exact, with checks at every third iteration."""
    hist = inputs.random_history(s, 2, h, seed=60 + 3 * h + s, swap=swap)
    start = [hist[1], hist[0]]  # oldest first
    _check_run_against_oracle(lb, orc, s, 2, h, 9, 3, 0, 0, start=start)


@pytest.mark.parametrize("s,h", D2S_SHAPES)
@pytest.mark.parametrize("r_mode", [0, 1])
def test_d2_swap_zero_start_every_iteration_checked(lb, orc, s, h, r_mode):
    """Zero start (swap-symmetric): the fused increment's argmin classes and the check, every iteration."""
    _check_run_against_oracle(lb, orc, s, 2, h, 12, 1, 0, r_mode)


@pytest.mark.parametrize("h", [4, 5, 6])
@pytest.mark.parametrize("perm", [False, True])
def test_d3_permutation_paths_bit_exact(lb, orc, h, perm):
    """sigma = 2, d = 3: starts symmetric under the string permutations (and
    the complement) run the kernels that read each orbit's values once; starts
    with the complement symmetry only run the generic kernels.  Both exact."""
    hist = inputs.random_history(2, 3, h, seed=90 + h, symmetric=True, swap=perm)
    start = [hist[2], hist[1], hist[0]]  # oldest first
    _check_run_against_oracle(lb, orc, 2, 3, h, 8, 3, 1, 0, start=start)


@pytest.mark.parametrize("h,r_mode", [(4, 0), (5, 1), (7, 0)])
def test_d3_permutation_zero_start_every_iteration_checked(lb, orc, h, r_mode):
    _check_run_against_oracle(lb, orc, 2, 3, h, 10, 1, 1, r_mode)


@pytest.mark.parametrize("h,perm", [(4, True), (5, True), (5, False)])
def test_d3_permutation_all_subsets_bit_exact(lb, orc, h, perm):
    """f_mode 1 (every non-empty advance set) through the permutation-aware
    kernels (symmetric starts) and the generic ones (complement only)."""
    hist = inputs.random_history(2, 3, h, seed=95 + h, symmetric=True, swap=perm)
    start = [hist[2], hist[1], hist[0]]
    _check_run_against_oracle(lb, orc, 2, 3, h, 8, 3, 1, 0, start=start, f_mode=1)


@pytest.mark.parametrize("h,r_mode", [(4, 0), (6, 1)])
def test_d3_permutation_all_subsets_zero_start(lb, orc, h, r_mode):
    _check_run_against_oracle(lb, orc, 2, 3, h, 10, 1, 1, r_mode, f_mode=1)


def test_d3_permutation_kernel_is_used_and_counted(lb):
    with lb.LcsBound(2, 3, 6, timing=1) as hnd:
        hnd.iterate(4)
        assert hnd.stats()["sweep_bytes"] == 4 * 15 * (8 ** 6 // 2)
    with lb.LcsBound(2, 3, 6, timing=1, f_mode=1) as hnd:
        hnd.iterate(4)
        assert hnd.stats()["sweep_bytes"] == 4 * 17 * (8 ** 6 // 2)


def test_d2_swap_kernel_is_used_and_counted(lb):
    with lb.LcsBound(3, 2, 6, timing=1) as hnd:
        hnd.iterate(5)
        st = hnd.stats()
        # 20 algorithmic bytes per state (v_{t-1} once, half of v_{t-2}, one write) instead of 8 (d+1) = 24
        assert st["sweep_bytes"] == 5 * 20 * 3 ** 12


@pytest.mark.parametrize("s,d,h,sym", [(2, 2, 5, 1), (2, 2, 5, 0), (2, 3, 3, 1), (3, 2, 3, 0), (4, 2, 2, 0),
                                       (3, 2, 4, 0), (4, 2, 3, 0)])
def test_check_vector_matches_oracle(lb, torch_mod, orc, s, d, h, sym):
    torch = torch_mod
    u = inputs.random_fx(s, d, h, seed=77 + h, symmetric=(s == 2))
    for R in [int(0.3 * (1 << K)), int(0.45 * (1 << K)), -(1 << 30)]:
        E_want, _ = orc.check(s, d, h, u, R, arith="fx")
        with lb.LcsBound(s, d, h, symmetry=sym) as hnd:
            E_got = hnd.check_vector(torch.from_numpy(u).cuda(), R)
        assert E_got == E_want


@pytest.mark.parametrize("h,printed", [(8, 0.776860), (9, 0.779259), (10, 0.781281)])
def test_binary_bound_matches_table2(lb, h, printed):
    """Table 2 (rounded down to 6 decimals) from the GPU path alone."""
    with lb.LcsBound(2, 2, h, check_every=50) as hnd:
        hnd.iterate(300)
        bound = hnd.read()[0]
    assert math.floor(bound * 1e6 + 1e-9) / 1e6 == pytest.approx(printed, abs=1e-9)


def test_bound_config_h8_matches_oracle(lb, orc):
    """(2,2,8), 200 iterations from zero: the same bound as the oracle, and Table 2's 0.776860."""
    want = orc.run(2, 2, 8, 200, arith="fx")
    with lb.LcsBound(2, 2, 8) as hnd:
        hnd.iterate(200)
        bound = hnd.read()[0]
        got_v = hnd.export_fx(0)
    assert bound == want["bound_rd"]
    assert np.array_equal(got_v, want["iterates"][0])
    assert math.floor(bound * 1e6 + 1e-9) / 1e6 == pytest.approx(0.776860, abs=1e-9)


def test_symmetric_and_full_storage_agree(lb):
    with lb.LcsBound(2, 2, 7, symmetry=1) as a, lb.LcsBound(2, 2, 7, symmetry=0) as b:
        assert a.n_stored * 2 == b.n_stored
        a.iterate(40)
        b.iterate(40)
        assert np.array_equal(a.export_fx(0), b.export_fx(0))
        assert a.read() == b.read()


def test_iterate_in_pieces_equals_one_call(lb):
    with lb.LcsBound(2, 3, 3, check_every=5) as a, lb.LcsBound(2, 3, 3, check_every=5) as b:
        a.iterate(23)
        for n in (7, 9, 7):
            b.iterate(n)
        assert np.array_equal(a.export_fx(0), b.export_fx(0))
        assert np.array_equal(a.export_fx(1), b.export_fx(1))


def test_double_roundtrip_and_export(lb, orc):
    s, d, h = 2, 2, 4
    with lb.LcsBound(s, d, h) as hnd:
        hnd.iterate(20)
        fx = hnd.export_fx(0)
        dbl = hnd.export(0)
        assert np.array_equal(dbl, fx.astype(np.float64) / 2.0 ** K)
        hnd.set_start([hnd.export(k) for k in range(d)])
        assert np.array_equal(hnd.export_fx(0), fx)


def test_device_pointer_start_and_export(lb, torch_mod):
    torch = torch_mod
    s, d, h = 2, 2, 5
    hist = inputs.random_history(s, d, h, seed=3, symmetric=True)
    with lb.LcsBound(s, d, h) as hnd:
        hnd.set_start_fx([torch.from_numpy(v).cuda() for v in hist])
        out = torch.empty(s ** (d * h), dtype=torch.int64, device="cuda")
        lb.lcs_bound_export_fx(hnd.hnd, 1, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), hist[1])


def test_errors(lb):
    with lb.LcsBound(2, 2, 3) as hnd:
        with pytest.raises(lb.LcsError) as e:
            hnd.read()
        assert e.value.status == 5  # LCS_ENOBOUND
        v = inputs.random_fx(2, 2, 3, seed=1)  # not complement-symmetric
        with pytest.raises(lb.LcsError) as e:
            hnd.set_start_fx([v, v])
        assert e.value.status == 1  # LCS_EINVAL
        with pytest.raises(lb.LcsError):
            hnd.iterate(-1)
        with pytest.raises(lb.LcsError) as e:
            hnd.export_fx(-1)  # u not retained
    with pytest.raises(lb.LcsError) as e:
        lb.LcsBound(11, 2, 2)  # the general kernels are compiled for sigma <= 10
    assert e.value.status == 7  # LCS_EUNSUPPORTED


def test_overflow_guard(lb):
    with lb.LcsBound(2, 2, 2, frac_bits=56) as hnd:
        with pytest.raises(lb.LcsError) as e:
            hnd.iterate(100)
        assert e.value.status == 6  # LCS_EOVERFLOW


def test_keep_u_retains_kept_iterate(lb, orc):
    s, d, h = 2, 2, 4
    want = orc.run(s, d, h, 30, arith="fx", check_every=4, want_u=True)
    with lb.LcsBound(s, d, h, check_every=4, keep_u=1) as hnd:
        hnd.iterate(30)
        assert np.array_equal(hnd.export_fx(-1), want["u"])


def test_torch_allocator_and_stream(lb, torch_mod):
    torch = torch_mod
    st = torch.cuda.Stream()
    with lb.LcsBound(2, 2, 6, torch_alloc=True, stream=st.cuda_stream) as a, lb.LcsBound(2, 2, 6) as b:
        a.iterate(30)
        b.iterate(30)
        assert np.array_equal(a.export_fx(0), b.export_fx(0))


def test_timing_stats(lb):
    n = 4 ** 6 // 2
    with lb.LcsBound(2, 2, 6, timing=1, check_every=10) as hnd:
        hnd.iterate(30)
        st = hnd.stats()
        # at h >= 6 the zero start runs the kernel that also uses the string
        # swap: 20 algorithmic bytes per stored state instead of 8 (d+1) = 24.
        # The checks of iterations 10 and 20 ran inside sweeps 11 and 21 (4
        # more bytes per stored state each); the check of iteration 30 waits
        # for the next sweep or for a call that reads results.
        assert st["sweep_launches"] == 30 and st["check_launches"] == 0
        assert st["sweep_ms"] > 0
        assert st["sweep_bytes"] == 30 * 20 * n + 2 * 4 * n
        hnd.read()
        st = hnd.stats()
        assert st["check_launches"] == 1 and st["check_ms"] > 0 and st["check_bytes"] == 8 * n
    with lb.LcsBound(2, 2, 5, timing=1, check_every=10) as hnd:  # no fused kernel: every check on its own
        hnd.iterate(30)
        st = hnd.stats()
        assert st["sweep_launches"] == 30 and st["check_launches"] == 3
        assert st["sweep_bytes"] == 30 * 24 * (4 ** 5 // 2)
        assert st["check_bytes"] == 3 * 8 * (4 ** 5 // 2)


# ---------------------------------------------------------------------------
# f_mode = 1: the max over every non-empty advance set (an extension the paper
# does not use; parity against the oracle's plain definition of it)

FALL_SHAPES = [(2, 2, 1), (2, 2, 4), (2, 3, 1), (2, 3, 3), (3, 2, 1), (3, 2, 3)]


@pytest.mark.parametrize("s,d,h", FALL_SHAPES)
def test_all_subsets_sweep_bit_exact(lb, torch_mod, orc, s, d, h):
    torch = torch_mod
    vs = inputs.random_history(s, d, h, seed=300 + 7 * h + d + s)
    want = orc.F(s, d, h, vs, arith="fx", f_mode=1)
    out = torch.empty(want.size, dtype=torch.int64, device="cuda")
    lb.lcs_sweep_fx(s, d, h, [torch.from_numpy(v).cuda() for v in vs], out, f_mode=1)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("s,d,h,sym", [(2, 2, 5, 1), (2, 2, 4, 0), (2, 3, 3, 1), (2, 3, 3, 0), (3, 2, 3, 0)])
def test_all_subsets_run_bit_exact(lb, orc, s, d, h, sym):
    iters, ce = 40, 7
    want = orc.run(s, d, h, iters, arith="fx", check_every=ce, f_mode=1)
    with lb.LcsBound(s, d, h, check_every=ce, symmetry=sym, f_mode=1) as hnd:
        hnd.iterate(iters)
        rep = hnd.report()
        for k in range(d):
            assert np.array_equal(hnd.export_fx(k), want["iterates"][k])
        assert (rep["R"], rep["argmin"], rep["E"], rep["r"], rep["eps"]) == (
            want["R"], want["argmin"], want["E"], want["r"], want["eps"])
        assert hnd.read()[0] == want["bound_rd"]
