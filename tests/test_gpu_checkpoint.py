"""Stored-form transfers and checkpoint/resume against an uninterrupted run.

A handle saved after some iterations and restored into a fresh handle must
continue bit for bit as the original does: same iterates, same R, argmin, E,
kept triplet and bound.  The stored form of an iterate is the prefix of the
full vector that the handle keeps (the states x < N/2 under complement
symmetry); a start given in that form must behave exactly as the same start
given in full.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return lb


SHAPES = [(2, 2, 7, {}), (3, 2, 3, {}), (2, 3, 4, {"keep_u": 1}), (2, 2, 5, {"symmetry": 0, "r_mode": 1})]


@pytest.mark.parametrize("s,d,h,kw", SHAPES)
def test_resume_continues_bit_for_bit(lb, tmp_path, s, d, h, kw):
    path = str(tmp_path / "ckpt.bin")
    with lb.LcsBound(s, d, h, check_every=7, **kw) as a:
        a.iterate(23)
        a.save(path)
        a.iterate(19)
        want = [a.export_fx(k) for k in range(d)]
        want_rep = a.report()
        want_read = a.read()
        want_u = a.export_fx(-1) if kw.get("keep_u") else None
    with lb.LcsBound(s, d, h, check_every=7, **kw) as b:
        b.iterate(3)  # whatever the handle held is replaced
        b.restore(path)
        b.iterate(19)
        for k in range(d):
            assert np.array_equal(b.export_fx(k), want[k]), k
        assert b.report() == want_rep
        assert b.read() == want_read
        if want_u is not None:
            assert np.array_equal(b.export_fx(-1), want_u)


def test_restore_rejects_other_shapes_and_bad_files(lb, tmp_path):
    path = str(tmp_path / "ckpt.bin")
    with lb.LcsBound(2, 2, 6, check_every=5) as a:
        a.iterate(10)
        a.save(path)
    for shape, kw in [((2, 2, 5), {}), ((2, 2, 6), {"check_every": 4}), ((2, 2, 6), {"symmetry": 0})]:
        kw = {"check_every": 5, **kw}
        with lb.LcsBound(*shape, **kw) as b:
            with pytest.raises(lb.LcsError) as e:
                b.restore(path)
            assert e.value.status == lb.LCS_EINVAL
    data = open(path, "rb").read()
    short = str(tmp_path / "short.bin")
    open(short, "wb").write(data[: len(data) // 2])
    junk = str(tmp_path / "junk.bin")
    open(junk, "wb").write(b"not a checkpoint" * 16)
    with lb.LcsBound(2, 2, 6, check_every=5) as b:
        with pytest.raises(lb.LcsError) as e:
            b.restore(short)
        assert e.value.status == lb.LCS_EIO
        with pytest.raises(lb.LcsError) as e:
            b.restore(junk)
        assert e.value.status == lb.LCS_EINVAL
        with pytest.raises(lb.LcsError) as e:
            b.restore(str(tmp_path / "missing.bin"))
        assert e.value.status == lb.LCS_EIO
        with pytest.raises(lb.LcsError) as e:
            b.save(str(tmp_path / "no_such_dir" / "x.bin"))
        assert e.value.status == lb.LCS_EIO


@pytest.mark.parametrize("s,d,h,sym", [(2, 2, 7, 1), (2, 3, 4, 1), (3, 2, 3, 0), (2, 2, 6, 0)])
def test_stored_form_round_trip(lb, s, d, h, sym):
    import torch

    with lb.LcsBound(s, d, h, check_every=10, symmetry=sym) as a:
        a.iterate(30)
        full = [a.export_fx(k) for k in range(d)]
        stored = [a.export_stored_fx(k) for k in range(d)]
        stored_dev = [torch.empty(a.n_stored, dtype=torch.int64, device="cuda") for _ in range(d)]
        for k in range(d):
            a.export_stored_fx(k, stored_dev[k])
        for k in range(d):
            assert stored[k].size == a.n_stored
            assert np.array_equal(stored[k], full[k][: a.n_stored])
            assert np.array_equal(stored_dev[k].cpu().numpy(), stored[k])
    with lb.LcsBound(s, d, h, check_every=10, symmetry=sym) as b, \
            lb.LcsBound(s, d, h, check_every=10, symmetry=sym) as c, \
            lb.LcsBound(s, d, h, check_every=10, symmetry=sym) as e:
        b.set_start_fx(full)
        c.set_start_stored_fx(stored)
        e.set_start_stored_fx(stored_dev)
        for hnd in (b, c, e):
            hnd.iterate(25)
        for k in range(d):
            assert np.array_equal(c.export_fx(k), b.export_fx(k))
            assert np.array_equal(e.export_fx(k), b.export_fx(k))
        assert c.read() == b.read() == e.read()


def _oracle_checks(orc, s, d, h, iters, check_every):
    """Algorithm 2 one iteration at a time: the record of every check the handle's cadence runs."""
    cur, kept, recs = None, {"r": 0, "eps": 0, "kept_iter": -1}, []
    for it in range(1, iters + 1):
        step = orc.run(s, d, h, 1, arith="fx", check_every=1, start=cur)
        if (check_every > 0 and it % check_every == 0) or it == iters:
            better = step["R"] - step["E"] >= kept["r"] - kept["eps"]
            if better:
                kept = {"r": step["R"], "eps": step["E"], "kept_iter": it}
            recs.append({"iter": it, "R": step["R"], "argmin": step["argmin"], "E": step["E"],
                         "kept": int(better), **kept})
        its = step["iterates"]
        cur = [its[d - 1 - k] for k in range(d)]
    return recs


@pytest.mark.parametrize("s,d,h", [(2, 2, 6), (3, 2, 3), (2, 3, 4)])
def test_check_history_matches_oracle(lb, orc, s, d, h):
    iters, ce = 23, 4
    want = _oracle_checks(orc, s, d, h, iters, ce)
    with lb.LcsBound(s, d, h, check_every=ce) as hnd:
        hnd.iterate(iters)
        recs, n = hnd.history()
    assert n == len(want)
    assert recs == want


def test_check_history_ring_and_resets(lb):
    with lb.LcsBound(2, 2, 3, check_every=1) as hnd:
        hnd.iterate(4100)
        recs, n = hnd.history(max_records=10)
        assert n == 4100 and [r["iter"] for r in recs] == list(range(4091, 4101))
        full, _ = hnd.history()
        assert len(full) == 4096 and full[0]["iter"] == 5 and full[-1] == recs[-1]
        hnd.set_start_fx([hnd.export_fx(0), hnd.export_fx(1)])
        assert hnd.history() == ([], 0)


def _orbit_reference(full, h):
    """The orbit form as the header defines it, rebuilt from a full vector
    with plain index arithmetic (the STATE INDEX of sigma = d = 2)."""
    K, M = 1 << (h - 2), (1 << (h - 1)) - 1

    def idx(g0, g1, a, b):
        x = (g0 << (2 * h - 1)) | (g1 << (2 * h - 2))
        for i in range(h - 1):
            x |= ((a >> i) & 1) << (2 * i + 1) | ((b >> i) & 1) << (2 * i)
        return x

    out = np.zeros(4 * K * (K + 1), dtype=np.int64)
    for s in (0, 1):
        for beta in range(K):
            b = beta if s == 0 else M - beta
            for a in range(beta + 1):
                q = s * (K * (K + 1) // 2) + beta * (beta + 1) // 2 + a
                out[4 * q:4 * q + 4] = [full[idx(0, 0, a, b)], full[idx(0, 0, M - a, M - b)],
                                        full[idx(0, 1, a, b)], full[idx(0, 1, M - a, M - b)]]
    return out


@pytest.mark.parametrize("h", [6, 7])
def test_orbit_form_layout_and_round_trip(lb, h):
    import torch

    d = 2
    with lb.LcsBound(2, d, h, check_every=10) as a:
        a.iterate(30)
        full = [a.export_fx(k) for k in range(d)]
        orb = [a.export_orbit_fx(k) for k in range(d)]
        orb_dev = [torch.empty(a.n_orbit, dtype=torch.int64, device="cuda") for _ in range(d)]
        for k in range(d):
            a.export_orbit_fx(k, orb_dev[k])
        assert a.n_orbit == 4 ** (h - 1) + 2 ** h
        for k in range(d):
            assert np.array_equal(orb[k], _orbit_reference(full[k], h)), k
            assert np.array_equal(orb_dev[k].cpu().numpy(), orb[k])
    with lb.LcsBound(2, d, h, check_every=10) as b, lb.LcsBound(2, d, h, check_every=10) as c, \
            lb.LcsBound(2, d, h, check_every=10) as e:
        b.set_start_fx(full)
        c.set_start_orbit_fx(orb)
        e.set_start_orbit_fx(orb_dev)
        for k in range(d):  # the start itself, all N states
            assert np.array_equal(c.export_fx(k), full[k])
            assert np.array_equal(e.export_fx(k), full[k])
        for hnd in (b, c, e):
            hnd.iterate(25)
        for k in range(d):
            assert np.array_equal(c.export_fx(k), b.export_fx(k))
            assert np.array_equal(e.export_fx(k), b.export_fx(k))
        assert c.read() == b.read() == e.read()


def test_orbit_form_errors(lb):
    import torch

    for shape, kw in [((2, 2, 5), {}), ((3, 2, 4), {}), ((2, 2, 7), {"symmetry": 0}), ((2, 3, 4), {})]:
        with lb.LcsBound(*shape, **kw) as hnd:
            with pytest.raises(lb.LcsError) as e:
                hnd.n_orbit
            assert e.value.status == lb.LCS_EUNSUPPORTED
    with lb.LcsBound(2, 2, 6) as hnd:
        n = hnd.n_orbit
        # a complement-symmetric start without the swap symmetry runs, but has no orbit form
        rng = np.random.default_rng(5)
        N = hnd.n_states
        v = rng.integers(0, 1 << 40, size=N, dtype=np.int64)
        v = np.minimum(v, v[::-1])
        hnd.set_start_fx([v, v])
        with pytest.raises(lb.LcsError) as e:
            hnd.export_orbit_fx(0)
        assert e.value.status == lb.LCS_EINVAL
        buf = torch.zeros(n + 2, dtype=torch.int64, device="cuda")
        with pytest.raises(lb.LcsError) as e:
            hnd.set_start_orbit_fx([buf[1:n + 1], buf[1:n + 1]])  # 8-byte aligned only
        assert e.value.status == lb.LCS_EINVAL


def test_orbit_form_of_the_kept_u(lb):
    h = 6
    with lb.LcsBound(2, 2, h, check_every=5, keep_u=1) as a:
        a.iterate(23)
        u_full = a.export_fx(-1)
        u_orb = a.export_orbit_fx(-1)
        assert np.array_equal(u_orb, _orbit_reference(u_full, h))
        with pytest.raises(lb.LcsError) as e:
            a.export_orbit_fx(2)  # k outside -1..d-1
        assert e.value.status == lb.LCS_EINVAL
    with lb.LcsBound(2, 2, h, check_every=5) as b:
        with pytest.raises(lb.LcsError) as e:
            b.export_orbit_fx(-1)  # u is not retained
        assert e.value.status == lb.LCS_EINVAL
