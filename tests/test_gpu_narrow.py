"""Offset-normalised 32-bit storage, the vector held in host memory (the
sweep running out of core) and the prefix-lift start.

32-bit storage keeps w = v - c with one offset c per vector.  Lemma 1's
translation invariance makes the mean of w + c the mean of w plus c, so the
iteration is the same integer recursion: iterates, R, argmin, E, the kept
triplet and the bound must equal the CPU oracle's fixed-point run at the same
number of fractional bits bit for bit, and so must every handle with one
vector in pinned host memory.  Overflow of the 32-bit range is made on
purpose from the host (too many fractional bits, no check) and must come back
as LCS_EOVERFLOW, never as a fault.
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return lb


def _result(hnd):
    rep = hnd.report()
    return (hnd.export_fx(0), hnd.export_fx(1), rep["R"], rep["argmin"], rep["E"], rep["r"], rep["eps"],
            rep["kept_iter"], hnd.read()[0])


def _same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2:] == b[2:]


@pytest.mark.parametrize("h,K,C,pieces,r_mode", [(6, 24, 5, [40], 0), (7, 26, 10, [13, 27], 1), (8, 24, 1, [30], 0),
                                                 (9, 25, 7, [20, 1, 9], 0)])
def test_narrow_zero_start_equals_oracle(lb, orc, h, K, C, pieces, r_mode):
    iters = sum(pieces)
    want = orc.run(2, 2, h, iters, arith="fx", frac_bits=K, check_every=C, r_mode=r_mode)
    with lb.LcsBound(2, 2, h, storage=1, frac_bits=K, check_every=C, r_mode=r_mode) as hnd:
        for n in pieces:
            hnd.iterate(n)
        got = _result(hnd)
    assert np.array_equal(got[0], want["iterates"][0]) and np.array_equal(got[1], want["iterates"][1])
    assert got[2:8] == (want["R"], want["argmin"], want["E"], want["r"], want["eps"], want["kept_iter"])
    assert got[8] == want["bound_rd"]


@pytest.mark.parametrize("h", [7, 10])
def test_narrow_random_start_equals_wide(lb, h):
    K = 24
    hist = inputs.random_history(2, 2, h, seed=h, frac_bits=K, symmetric=True, swap=True)
    stored = [v[: v.size // 2].copy() for v in hist]
    results = []
    for kw in ({}, {"storage": 1}):
        with lb.LcsBound(2, 2, h, frac_bits=K, check_every=4, **kw) as hnd:
            hnd.set_start_stored_fx(stored)
            hnd.iterate(10)
            hnd.iterate(7)
            results.append(_result(hnd))
            st = hnd.export_stored_fx(0)
            assert np.array_equal(st, results[-1][0][: st.size])
    _same(results[0], results[1])


@pytest.mark.parametrize("h", [10, 12])
@pytest.mark.parametrize("storage", [0, 1])
def test_host_slot_equals_device_only(lb, h, storage):
    """One of the three vectors in pinned host memory: the sweeps that read or
    write it go over the host link, with the same results bit for bit."""
    K = 26
    with lb.LcsBound(2, 2, h, frac_bits=K, check_every=10) as ref:
        ref.iterate(31)
        want = _result(ref)
    with lb.LcsBound(2, 2, h, frac_bits=K, check_every=10, storage=storage, host_slots=1) as hnd:
        hnd.iterate(31)
        got = _result(hnd)
    _same(got, want)


def test_host_slot_general_kernels(lb, orc):
    """The host-resident vector is plain memory to every kernel family."""
    s, d, h, K = 3, 2, 3, 36
    want = orc.run(s, d, h, 20, arith="fx", frac_bits=K, check_every=5)
    with lb.LcsBound(s, d, h, frac_bits=K, check_every=5, host_slots=1) as hnd:
        hnd.iterate(20)
        assert np.array_equal(hnd.export_fx(0), want["iterates"][0])
        assert hnd.read()[0] == want["bound_rd"]


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("on_device", [False, True])
def test_lift_start_equals_explicit_lift(lb, storage, on_device):
    import torch

    K, h_from, h = 26, 8, 10
    with lb.LcsBound(2, 2, h_from, frac_bits=K, check_every=50) as small:
        small.iterate(150)
        src = small.export_stored_fx(0)
        r_hat = small.report()["r"]
    s2 = 2 * (h - h_from)
    x = np.arange(4 ** h // 2)
    newest = src[x >> s2]
    explicit = [newest, newest - r_hat]
    with lb.LcsBound(2, 2, h, frac_bits=K, check_every=5) as ref:
        ref.set_start_stored_fx(explicit)
        ref.iterate(12)
        want = _result(ref)
    with lb.LcsBound(2, 2, h, frac_bits=K, check_every=5, storage=storage) as hnd:
        hnd.set_start_lift_fx(h_from, torch.from_numpy(src).cuda() if on_device else src, r_hat)
        assert np.array_equal(hnd.export_stored_fx(0), newest)
        assert np.array_equal(hnd.export_stored_fx(1), newest - r_hat)
        hnd.iterate(12)
        got = _result(hnd)
    _same(got, want)


def test_narrow_overflow_is_reported(lb):
    """30 fractional bits leave 32-bit rows +-2 units around their offset.  A
    start whose rows fit (newest all 0, older all 1.9 units) gives equal-head
    states 1 + 1.9 units in one sweep, while the output's offset is anchored at
    the newest value of state 0 (0, no increment yet): 2.9 units do not fit,
    and the sweep must say so."""
    K = 30
    n = 4 ** 6 // 2
    newest = np.zeros(n, dtype=np.int64)
    older = np.full(n, int(1.9 * (1 << K)), dtype=np.int64)
    with lb.LcsBound(2, 2, 6, storage=1, frac_bits=K, check_every=0) as hnd:
        hnd.set_start_stored_fx([newest, older])
        hnd.iterate(1)
        with pytest.raises(lb.LcsError) as e:
            hnd.read()
        assert e.value.status == lb.LCS_EOVERFLOW
    with lb.LcsBound(2, 2, 6, frac_bits=K, check_every=0) as wide:  # the same start in 64 bits runs
        wide.set_start_stored_fx([newest, older])
        wide.iterate(1)
        wide.read()
    # a start whose spread exceeds the range is refused
    K = 30
    v = inputs.random_fx(2, 2, 6, seed=3, spread_units=40.0, frac_bits=K, symmetric=True, swap=True)
    with lb.LcsBound(2, 2, 6, storage=1, frac_bits=K) as hnd:
        with pytest.raises(lb.LcsError) as e:
            hnd.set_start_stored_fx([v[: v.size // 2]] * 2)
        assert e.value.status == lb.LCS_EOVERFLOW


def test_narrow_refusals(lb):
    import torch

    for kw, status in [({"frac_bits": 44}, lb.LCS_EINVAL), ({"keep_u": 1, "frac_bits": 24}, lb.LCS_EUNSUPPORTED),
                       ({"symmetry": 0, "frac_bits": 24}, lb.LCS_EUNSUPPORTED), ({"host_slots": 2}, lb.LCS_EINVAL)]:
        with pytest.raises(lb.LcsError) as e:
            lb.LcsBound(2, 2, 8, storage=1, **kw)
        assert e.value.status == status, kw
    with pytest.raises(lb.LcsError) as e:
        lb.LcsBound(3, 2, 4, storage=1, frac_bits=24)
    assert e.value.status == lb.LCS_EUNSUPPORTED
    with lb.LcsBound(2, 2, 8, storage=1, frac_bits=24, check_every=5) as hnd:
        hnd.iterate(5)
        for call in (lambda: hnd.n_orbit, lambda: hnd.save("/tmp/never_written.bin"),
                     lambda: hnd.check_vector(torch.zeros(hnd.n_stored, dtype=torch.int64, device="cuda"), 0),
                     lambda: hnd.set_start_fx([np.zeros(hnd.n_states, dtype=np.int64)] * 2)):
            with pytest.raises(lb.LcsError) as e:
                call()
            assert e.value.status == lb.LCS_EUNSUPPORTED
        # a start without the swap symmetry
        v = inputs.random_fx(2, 2, 8, seed=5, frac_bits=24, symmetric=True)
        with pytest.raises(lb.LcsError) as e:
            hnd.set_start_stored_fx([v[: v.size // 2]] * 2)
        assert e.value.status == lb.LCS_EINVAL


def test_host_buffer_round_trip(lb):
    """lcs_host_alloc's memory serves as a host vector for starts and exports."""
    h = 8
    with lb.LcsBound(2, 2, h, check_every=10) as a, lb.HostBuffer(4 ** h // 2) as buf:
        a.iterate(30)
        a.export_stored_fx(0, out=buf.array)
        assert np.array_equal(buf.array, a.export_stored_fx(0))
        with lb.LcsBound(2, 2, h, check_every=10) as b:
            b.set_start_stored_fx([buf.array, buf.array])
            b.iterate(5)
            b.read()
