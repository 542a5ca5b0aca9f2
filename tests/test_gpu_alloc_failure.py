"""Allocation failure, injected on the host: an allocator callback that
returns NULL at its k-th call.

For every k up to the number of device allocations a creation makes, the
creation must return LCS_ENOMEM with no handle and free everything it had
allocated (the callback's count of live allocations returns to zero).  The
same holds for the batch and the warm-start network, and for the buffers a
handle allocates on first use (the staging buffers of host transfers, the
network's training buffers).  No GPU fault is involved: the failure is a
NULL from the host callback.
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


def _failing_allocator(lb, fail_at):
    """TorchAllocator whose fail_at-th call (1-based; 0 = never) returns NULL; counts its calls."""

    class Failing(lb.TorchAllocator):
        def __init__(self):
            super().__init__()
            self.calls = 0

        def _alloc(self, nbytes, ctx):
            self.calls += 1
            if self.calls == fail_at:
                return None
            return super()._alloc(nbytes, ctx)

    return Failing()


def _opts(lb, a, **kw):
    o = lb.lcs_bound_default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    o.alloc, o.free = a.alloc, a.free
    return o


CASES = [((2, 2, 8), {}), ((2, 2, 8), {"keep_u": 1}), ((3, 2, 4), {}), ((2, 3, 4), {"symmetry": 0}),
         ((3, 8, 1), {"frac_bits": 30}), ((3, 4, 2), {"frac_bits": 36})]


@pytest.mark.parametrize("shape,kw", CASES, ids=lambda v: str(v))
def test_create_fails_cleanly_at_every_allocation(lb, shape, kw):
    ok = _failing_allocator(lb, 0)
    h = lb.lcs_bound_create(*shape, _opts(lb, ok, **kw))
    n_alloc = ok.calls
    assert n_alloc >= 5 and len(ok._live) == n_alloc
    lb.lcs_bound_destroy(h)
    assert len(ok._live) == 0
    for k in range(1, n_alloc + 1):
        a = _failing_allocator(lb, k)
        with pytest.raises(lb.LcsError) as e:
            lb.lcs_bound_create(*shape, _opts(lb, a, **kw))
        assert e.value.status == lb.LCS_ENOMEM, (k, e.value)
        assert a.calls >= k and len(a._live) == 0, (k, a.calls, len(a._live))


def test_staging_allocation_failure_keeps_the_handle(lb):
    """The staging buffers of a host transfer are allocated on first use: when
    that fails, set_start returns LCS_ENOMEM and the handle stays usable."""
    ok = _failing_allocator(lb, 0)
    h = lb.lcs_bound_create(2, 2, 6, _opts(lb, ok))
    n_create = ok.calls
    lb.lcs_bound_destroy(h)
    a = _failing_allocator(lb, n_create + 1)
    h = lb.lcs_bound_create(2, 2, 6, _opts(lb, a, check_every=5))
    v = np.zeros(4 ** 6)
    with pytest.raises(lb.LcsError) as e:
        lb.lcs_bound_set_start(h, [v, v])  # full vectors from the host: converted through staging
    assert e.value.status == lb.LCS_ENOMEM
    lb.lcs_bound_set_start(h, [v, v])  # the next attempt allocates again and succeeds
    lb.lcs_bound_iterate(h, 10)
    got = lb.lcs_bound_read(h)
    lb.lcs_bound_destroy(h)
    assert len(a._live) == 0
    with lb.LcsBound(2, 2, 6, check_every=5) as plain:
        plain.iterate(10)
        assert plain.read() == got


def test_batch_create_fails_cleanly_at_every_allocation(lb):
    shapes = [(2, 2, 6), (3, 2, 3), (2, 3, 3), (2, 4, 2), (4, 2, 2)]
    ok = _failing_allocator(lb, 0)
    h = lb.lcs_bound_batch_create(shapes, _opts(lb, ok))
    n_alloc = ok.calls
    assert n_alloc >= len(shapes) * 3
    lb.lcs_bound_destroy(h)
    assert len(ok._live) == 0
    for k in range(1, n_alloc + 1):
        a = _failing_allocator(lb, k)
        with pytest.raises(lb.LcsError) as e:
            lb.lcs_bound_batch_create(shapes, _opts(lb, a))
        assert e.value.status == lb.LCS_ENOMEM, (k, e.value)
        assert len(a._live) == 0, (k, len(a._live))


def test_mlp_allocation_failures(lb):
    import torch

    ok = _failing_allocator(lb, 0)
    m = lb.LcsMlp(seed=3, allocator=ok)
    n_create = ok.calls
    assert n_create == 5
    m.close()
    assert len(ok._live) == 0
    for k in range(1, n_create + 1):
        a = _failing_allocator(lb, k)
        with pytest.raises(lb.LcsError) as e:
            lb.LcsMlp(seed=3, allocator=a)
        assert e.value.status == lb.LCS_ENOMEM
        assert len(a._live) == 0
    # the training buffers (made by the first gradient call): a failure leaves a usable handle
    states = np.arange(64, dtype=np.int64)
    hs = np.full(64, 4, dtype=np.int32)
    targets = np.linspace(-1, 1, 64).astype(np.float32)
    a = _failing_allocator(lb, n_create + 3)
    m = lb.LcsMlp(seed=3, allocator=a)
    with pytest.raises(lb.LcsError) as e:
        m.gradient(states, hs, targets)
    assert e.value.status == lb.LCS_ENOMEM
    loss, g = m.gradient(states, hs, targets)
    assert np.isfinite(loss) and np.all(np.isfinite(g))
    m.close()
    assert len(a._live) == 0
    # the inference table (made by the first bf16 prediction): the same
    a = _failing_allocator(lb, n_create + 1)
    m = lb.LcsMlp(seed=3, allocator=a)
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(lb.LcsError) as e:
        m.predict_bf16(4, 0, 16, out)
    assert e.value.status == lb.LCS_ENOMEM
    m.predict_bf16(4, 0, 16, out)
    assert torch.isfinite(out).all()
    m.close()
    assert len(a._live) == 0
