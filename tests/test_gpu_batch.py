"""Batched instances: every instance of a batch, bit for bit, against the oracle.

Mode 0: all instances advance in lockstep inside one cooperative persistent
kernel (captured in a CUDA graph).  Mode 1: each instance's single-instance
kernels run on a stream of its own.  In both, each instance must produce
exactly what Algorithm 2 gives for it alone.  The grid barrier's timeout path is exercised with a zero clock
budget: the launch must end with LCS_ETIMEOUT, not hang.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ETIMEOUT = 4


@pytest.fixture(scope="module")
def lb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return lb


MIXED = [(2, 2, 3), (2, 2, 6), (3, 2, 2), (4, 2, 2), (2, 3, 2), (2, 4, 2), (2, 2, 7), (3, 2, 3)]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("check_every,pieces", [(0, [17]), (5, [7, 9, 1]), (1, [6]), (5, [5, 5, 5, 5, 5, 5])])
def test_batch_matches_oracle(lb, orc, check_every, pieces, mode):
    iters = sum(pieces)
    with lb.LcsBatch(MIXED, check_every=check_every) as b:
        b.set_mode(mode)
        assert b.info()["mode"] == mode
        for n in pieces:
            b.iterate(n)
        for i, (s, d, h) in enumerate(MIXED):
            # the oracle checks at multiples of check_every and at the last
            # iteration of each call: run it call by call with the same cadence
            want = _oracle_in_pieces(orc, s, d, h, pieces, check_every)
            rep = b.report(i)
            assert rep["status"] == 0
            assert rep["iters_done"] == iters
            for k in range(d):
                assert np.array_equal(b.export_fx(i, k), want["iterates"][k]), (i, k)
            assert (rep["R"], rep["argmin"], rep["E"]) == (want["R"], want["argmin"], want["E"]), i
            assert (rep["r"], rep["eps"], rep["kept_iter"]) == (want["r"], want["eps"], want["kept_iter"]), i
            assert b.read(i)[0] == want["bound_rd"]


def _oracle_in_pieces(orc, s, d, h, pieces, check_every):
    """Algorithm 2 with checks at it % check_every == 0 and at the end of every piece.

    The oracle is stepped one iteration at a time (each step checked) and only
    the checks of the library's cadence enter the kept triplet.
    """
    ends = set(np.cumsum(pieces).tolist())
    cur = None  # zero start
    kept = {"r": 0, "eps": 0, "kept_iter": -1}
    last = None
    for it in range(1, sum(pieces) + 1):
        step = orc.run(s, d, h, 1, arith="fx", check_every=1, start=cur)
        if (check_every > 0 and it % check_every == 0) or it in ends:
            if step["R"] - step["E"] >= kept["r"] - kept["eps"]:
                kept = {"r": step["R"], "eps": step["E"], "kept_iter": it}
            last = step
        its = step["iterates"]  # newest first
        cur = [its[d - 1 - k] for k in range(d)]  # oldest first, as the oracle takes a start
    out = {"R": last["R"], "argmin": last["argmin"], "E": last["E"], "iterates": its}
    out.update(kept)
    out["bound_rd"] = orc.fx_to_double_rd(d * (kept["r"] - kept["eps"]))
    return out


@pytest.mark.parametrize("mode", [None, 0, 1, 2])
def test_batch_config3_shapes_match_single_handles(lb, mode):
    """The eight-instance benchmark batch against the validated single-instance
    path, in the autotuner's mode and in each mode forced."""
    shapes = [(2, 2, 10), (2, 2, 12), (3, 2, 6), (3, 2, 7), (4, 2, 5), (2, 3, 6), (2, 3, 7), (2, 4, 5)]
    iters = 60
    with lb.LcsBatch(shapes, check_every=20) as b:
        if mode is not None:
            b.set_mode(mode)
        b.iterate(iters)
        info = b.info()
        assert info["n_instances"] == 8 and info["grid"] > 0
        assert info["persistent_ms_per_iter"] > 0 and info["concurrent_ms_per_iter"] > 0
        if mode is None:
            assert info["mode"] == (1 if info["concurrent_ms_per_iter"] < info["persistent_ms_per_iter"] else 0)
        assert info["min_ctas_per_sm"] in (2, 4)
        total = iters
        if mode in (0, 1, 2):
            # a second call of the same length: mode 0 replays the graph of the
            # persistent launch it captured; mode 1 captures this call's
            # schedule (the ring slots and the check phase repeat after 60
            # iterations) and replays it; mode 2 never captures
            b.iterate(iters)
            total += iters
            info = b.info()
            if mode == 0:
                assert info["graph_captured"] == 1 and info["graph"] == 1 and info["graph_replays"] >= 1
            elif mode == 1:
                assert info["mode"] == 1 and info["graph_captured"] == 1 and info["graph_replays"] >= 1
            else:
                assert info["graph_captured"] == 0 and info["graph_replays"] == 0
        for i, (s, d, h) in enumerate(shapes):
            with lb.LcsBound(s, d, h, check_every=20) as one:
                one.iterate(total)
                assert np.array_equal(b.export_fx(i, 0), one.export_fx(0)), i
                assert b.read(i) == one.read(), i


def test_batch_barrier_timeout_reports_status(lb):
    """A zero clock budget makes every waiting CTA give up: LCS_ETIMEOUT, and the context stays usable."""
    with lb.LcsBatch([(2, 2, 8), (3, 2, 3)]) as b:
        b.set_mode(0)
        b.set_spin_budget(0)
        b.iterate(3)
        rep = b.report(0)
        assert rep["status"] == ETIMEOUT
        with pytest.raises(lb.LcsError) as e:
            b.read(0)
        assert e.value.status == ETIMEOUT
    # the device still works: a fresh run reaches the paper's bound for (2,2,6)
    with lb.LcsBound(2, 2, 6) as one:
        one.iterate(200)
        assert abs(one.read()[0] - 0.770273) < 1e-6


def test_batch_mode_is_fixed_once_iterating(lb):
    with lb.LcsBatch([(2, 2, 6), (3, 2, 2)]) as b:
        b.iterate(2)
        with pytest.raises(lb.LcsError) as e:
            b.set_mode(0)
        assert e.value.status == 1


def test_batch_rejects_unsupported(lb):
    with pytest.raises(lb.LcsError) as e:
        lb.LcsBatch([(5, 2, 2)])
    assert e.value.status == 7
    with pytest.raises(lb.LcsError) as e:
        lb.LcsBatch([(2, 2, 3)] * 17)
    assert e.value.status == 1
