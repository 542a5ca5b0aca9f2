"""The warm-start network's GPU kernels against the CPU reference, and the warm start itself.

The forward and backward kernels are checked against oracle/mlp.py (float64)
on random batches; FP32 accumulation differs from float64 by rounding only,
so gradients must agree to 2e-3 of their scale.  The warm start must give
the same rigorous bound as the zero start (the check decides the bound), and
its effect on the iteration count is reported, whatever it is.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return lb


def _unflatten(flat):
    H, F = omlp.HIDDEN, omlp.N_FEAT
    o = 0
    out = {}
    for name, shape in [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", ())]:
        size = int(np.prod(shape)) if shape else 1
        out[name] = flat[o:o + size].astype(np.float64).reshape(shape) if shape else np.array(float(flat[o]))
        o += size
    return out


def _flatten(g):
    return np.concatenate([np.asarray(g[k], dtype=np.float64).reshape(-1) for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def _batch(seed, n=96):
    rng = np.random.default_rng(seed)
    hs = rng.integers(3, 15, size=n)
    states = np.array([rng.integers(0, 1 << (2 * int(h))) for h in hs], dtype=np.int64)
    t = rng.normal(0, 2, size=n).astype(np.float32)
    return states, hs.astype(np.int32), t


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_reference(lb, seed):
    with lb.LcsMlp(seed=seed) as m:
        flat = m.get_params()
        states, hs, t = _batch(seed)
        loss, g = m.gradient(states, hs, t)
        P = _unflatten(flat)
        X = np.concatenate([omlp.features(states[i:i + 1], int(hs[i])) for i in range(states.size)])
        loss_ref, g_ref = omlp.loss_and_grads(P, X, t.astype(np.float64))
        gr = _flatten(g_ref)
        assert abs(loss - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref))
        assert np.max(np.abs(g - gr)) <= 2e-3 * np.max(np.abs(gr)) + 1e-7


def test_predict_matches_reference(lb):
    import torch

    with lb.LcsMlp(seed=5) as m:
        P = _unflatten(m.get_params())
        h = 9
        rng = np.random.default_rng(0)
        states = rng.integers(0, 1 << (2 * h), size=3000).astype(np.int64)
        out = torch.empty(states.size, dtype=torch.float32, device="cuda")
        m.predict(h, torch.from_numpy(states).cuda(), out)
        torch.cuda.synchronize()
        y_ref, _ = omlp.forward(P, omlp.features(states, h))
        assert np.max(np.abs(out.cpu().numpy() - y_ref)) <= 1e-4 * max(1.0, np.max(np.abs(y_ref)))


@pytest.mark.parametrize("h,base,n", [(1, 0, 4), (5, 0, 4 ** 5), (9, 0, 4 ** 9), (12, 123456, 5000),
                                      (14, 3 * 4 ** 13 + 777, 6000), (16, 4 ** 16 - 4096, 4096)])
def test_predict_bf16_matches_reference(lb, h, base, n):
    """Tensor-core inference (one fused kernel per prediction table, then a
    gather) against the float64 network with the same two bf16 roundings,
    and loosely against the unrounded network."""
    import torch

    with lb.LcsMlp(seed=7) as m:
        P = _unflatten(m.get_params())
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        m.predict_bf16(h, base, n, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(h)
    idx = np.unique(np.concatenate([rng.integers(0, n, size=min(n, 2500)), [0, n - 1]]))
    states = base + idx.astype(np.int64)
    X = omlp.features(states, h)
    y_bf16 = omlp.forward_bf16(P, X)
    y_ref, _ = omlp.forward(P, X)
    scale = max(1e-3, float(np.max(np.abs(y_ref))))
    err = np.abs(got[idx] - y_bf16)
    # most rows differ by the fp32 accumulation order only; a first-layer
    # activation whose fp32 and float64 values straddle a bf16 rounding
    # boundary rounds one ulp (2^-8 relative) apart, which moves y by up to
    # about 2^-8 |a| sum_j |w3_j W2_jk| ~ 5e-4 of its scale
    assert np.median(err) <= 1e-6 * scale
    assert np.max(err) <= 1e-3 * scale
    assert np.max(np.abs(got[idx] - y_ref)) <= 2e-2 * scale


def test_start_vectors_are_the_table_and_symmetric(lb):
    """The start has the iterate's symmetries exactly and newest - older = r_hat."""
    import torch

    h, r_hat = 10, 0.390625
    n = 4 ** h
    with lb.LcsMlp(seed=8) as m:
        newest = torch.empty(n, dtype=torch.float64, device="cuda")
        older = torch.empty(n, dtype=torch.float64, device="cuda")
        m.start_vectors(h, r_hat, newest, older)
        pred = torch.empty(n, dtype=torch.float32, device="cuda")
        m.predict_bf16(h, 0, n, pred)
        torch.cuda.synchronize()
    o = older.cpu().numpy()
    assert np.array_equal(o, pred.cpu().numpy().astype(np.float64))
    assert np.array_equal(newest.cpu().numpy(), o + r_hat)
    x = np.arange(n, dtype=np.int64)
    comp = (n - 1) - x
    swap = ((x >> 1) & 0x5555555555555555) | ((x & 0x5555555555555555) << 1)
    assert np.array_equal(o[comp], o)
    assert np.array_equal(o[swap], o)


def _converged(lb, h, iters=300):
    import torch

    with lb.LcsBound(2, 2, h, check_every=50) as hnd:
        hnd.iterate(iters)
        v = torch.empty(4 ** h, dtype=torch.int64, device="cuda")
        lb.lcs_bound_export_fx(hnd.hnd, 0, v)
        return v, hnd.read()


def test_training_reduces_loss_and_warm_start_keeps_the_bound(lb):
    import torch

    data = {h: _converged(lb, h) for h in (5, 6, 7)}
    with lb.LcsMlp(seed=11) as m:
        vecs = [data[h][0] for h in (5, 6, 7)]
        before = m.train(vecs, [5, 6, 7], steps=0, batch=2048)
        after = m.train(vecs, [5, 6, 7], steps=400, batch=2048, lr=2e-3)
        assert after < 0.25 * before
        h = 8
        r_hat = data[7][1][2]  # r of the h = 7 run
        newest = torch.empty(4 ** h, dtype=torch.float64, device="cuda")
        older = torch.empty(4 ** h, dtype=torch.float64, device="cuda")
        m.start_vectors(h, r_hat, newest, older)
    with lb.LcsBound(2, 2, h, check_every=10) as zero, lb.LcsBound(2, 2, h, check_every=10) as warm:
        warm.set_start([newest, older])
        zero.iterate(400)
        warm.iterate(400)
        bz, bw = zero.read()[0], warm.read()[0]
    # both rigorous; both converge to Table 2's 0.776860 for h = 8
    assert abs(bz - bw) < 1e-7
    assert abs(bw - 0.776860) < 1e-6


def test_lift_prefix_cuts_tuples(lb):
    """The non-learned control: the value of a tuple is that of its first h_from letters, relative to state 0."""
    import torch

    h_from, h_to, r_hat = 4, 6, 0.375
    rng = np.random.default_rng(2)
    src = rng.integers(-(1 << 50), 1 << 50, size=4 ** h_from, dtype=np.int64)
    newest = torch.empty(4 ** h_to, dtype=torch.float64, device="cuda")
    older = torch.empty(4 ** h_to, dtype=torch.float64, device="cuda")
    lb.lcs_lift_prefix(h_from, h_to, torch.from_numpy(src).cuda(), r_hat, newest, older)
    x = np.arange(4 ** h_to)
    want = (src[x >> (2 * (h_to - h_from))] - src[0]).astype(np.float64) * 2.0 ** -44
    assert np.array_equal(older.cpu().numpy(), want)
    assert np.array_equal(newest.cpu().numpy(), want + r_hat)


def test_stored_fixed_point_start_equals_the_double_start(lb):
    """The stored-form fixed-point start is the double start converted as set_start converts it."""
    import torch

    h, r_hat = 10, 0.3906
    n = 4 ** h
    with lb.LcsMlp(seed=9) as m:
        newest = torch.empty(n, dtype=torch.float64, device="cuda")
        older = torch.empty(n, dtype=torch.float64, device="cuda")
        m.start_vectors(h, r_hat, newest, older)
        nf = torch.empty(n // 2, dtype=torch.int64, device="cuda")
        of = torch.empty(n // 2, dtype=torch.int64, device="cuda")
        m.start_vectors_stored_fx(h, r_hat, nf, of)
        torch.cuda.synchronize()
    scale = 2.0 ** 44
    assert np.array_equal(nf.cpu().numpy(), np.floor(newest.cpu().numpy()[: n // 2] * scale).astype(np.int64))
    assert np.array_equal(of.cpu().numpy(), np.floor(older.cpu().numpy()[: n // 2] * scale).astype(np.int64))
    with lb.LcsBound(2, 2, h, check_every=10) as a, lb.LcsBound(2, 2, h, check_every=10) as b:
        a.set_start([newest, older])
        b.set_start_stored_fx([nf, of])
        a.iterate(30)
        b.iterate(30)
        assert np.array_equal(a.export_fx(0), b.export_fx(0))
        assert a.read() == b.read()


def _iterations_to(lb, H, target, start=None, limit=400):
    """iterations of Algorithm 2 (a check after every one) until the bound reaches target"""
    with lb.LcsBound(2, 2, H, check_every=1) as hnd:
        if start is not None:
            hnd.set_start(start)
        for it in range(1, limit + 1):
            hnd.iterate(1)
            if hnd.read()[0] >= target:
                return it
    return None


def test_learned_start_reaches_the_bound_in_fewer_iterations(lb):
    """What the trained network gains: iterations until the bound comes within
    1e-7 of the zero start's converged bound at h = 10, from the zero start
    (the method), from the prefix-truncation lift of h = 8 (the non-learned
    control) and from the network trained on the converged iterates of
    h = 6, 7, 8.  The learned start must need fewer iterations than the zero
    start; all three reach the same rigorous bound (Lemma 1: the check
    decides it)."""
    import torch

    H, train_h = 10, (6, 7, 8)
    ref = _converged(lb, H, iters=2000)[1][0]
    target = ref - 1e-7
    it_zero = _iterations_to(lb, H, target)
    data = {h: _converged(lb, h, iters=1000) for h in train_h}
    r_hat = data[max(train_h)][1][2]
    newest = torch.empty(4 ** H, dtype=torch.float64, device="cuda")
    older = torch.empty(4 ** H, dtype=torch.float64, device="cuda")
    lb.lcs_lift_prefix(max(train_h), H, data[max(train_h)][0], r_hat, newest, older)
    it_lift = _iterations_to(lb, H, target, [newest, older])
    with lb.LcsMlp(seed=2024) as m:
        m.train([data[h][0] for h in train_h], list(train_h), steps=1000, batch=4096, lr=1e-3)
        m.start_vectors(H, r_hat, newest, older)
    it_mlp = _iterations_to(lb, H, target, [newest, older])
    print(f"h = {H}: iterations to the bound - 1e-7: zero start {it_zero}, prefix lift {it_lift}, learned {it_mlp}")
    assert it_zero is not None and it_lift is not None and it_mlp is not None
    assert it_mlp < it_zero
