"""The entry point that allocates nothing, against the handle API.

lcs_sweep_incr_fx_noalloc serves callers that cannot allocate device memory
(code inside a memory pool it does not own, plugins whose host forbids
allocations, processes that have committed all free HBM): its reduction
scratch is a fixed array inside the library.  It must produce what a handle
produces for one checked iteration -- the new iterate, R and its state -- on
consecutive calls that share that array.  Results are integers: compared
exactly.  This file is collected last.
"""
import gc

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return torch, lb


def _via_handle(lb, s, d, h, hist, r_mode):
    with lb.LcsBound(s, d, h, symmetry=0, r_mode=r_mode) as hnd:
        hnd.set_start_fx(hist)
        hnd.iterate(1)
        rep = hnd.report()
        return hnd.export_fx(0), rep["R"], rep["argmin"]


def _via_noalloc(torch, lb, s, d, h, hist, r_mode):
    dev = [torch.from_numpy(v).cuda() for v in hist]
    out = torch.empty(s ** (d * h), dtype=torch.int64, device="cuda")
    R = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    arg = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    lb.lcs_sweep_incr_fx_noalloc(s, d, h, dev, out, R, arg, r_mode=r_mode)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(R.item()), int(arg.item())


def test_noalloc_matches_handle_on_consecutive_calls(env):
    torch, lb = env
    # a larger shape first, then a smaller one that launches fewer CTAs, then a
    # different kernel: each call must ignore whatever the previous left behind
    cases = [(2, 2, 7, 0, 11), (2, 2, 4, 0, 12), (3, 2, 3, 1, 13)]
    for s, d, h, r_mode, seed in cases:
        hist = inputs.random_history(s, d, h, seed=seed)
        want_v, want_R, want_arg = _via_handle(lb, s, d, h, hist, r_mode)
        got_v, got_R, got_arg = _via_noalloc(torch, lb, s, d, h, hist, r_mode)
        assert np.array_equal(got_v, want_v)
        assert (got_R, got_arg) == (want_R, want_arg)


def test_noalloc_rejects_bad_arguments(env):
    torch, lb = env
    v = torch.zeros(16, dtype=torch.int64, device="cuda")
    R = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lb.LcsError) as e:
        lb.lcs_sweep_incr_fx_noalloc(2, 2, 2, [v, v], v, R, R)
    assert e.value.status == 1  # output aliases an input
    # an output that is an offset view of an input: shares all but one value
    big = torch.zeros(17, dtype=torch.int64, device="cuda")
    A = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(lb.LcsError) as e:
        lb.lcs_sweep_incr_fx_noalloc(2, 2, 2, [big[:16], big[:16]], big[1:], R, A)
    assert e.value.status == 1


def test_noalloc_allocates_nothing_and_runs_on_a_caller_stream(env):
    """The property the entry point exists for: after a first call (which may
    load the library's device code), further calls change neither the
    device's free memory nor PyTorch's allocations, here on a caller-owned
    stream, and their results still equal the handle's."""
    torch, lb = env
    s, d, h = 2, 2, 6
    hist = inputs.random_history(s, d, h, seed=21)
    want_v, want_R, want_arg = _via_handle(lb, s, d, h, hist, 0)
    dev = [torch.from_numpy(v).cuda() for v in hist]
    out = torch.empty(s ** (d * h), dtype=torch.int64, device="cuda")
    R = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    arg = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    lb.lcs_sweep_incr_fx_noalloc(s, d, h, dev, out, R, arg, stream=stream.cuda_stream)  # warm-up
    stream.synchronize()
    gc.collect()  # tensors of earlier tests are freed now, not in the middle of the checks
    for _ in range(3):
        out.fill_(0)
        R.fill_(-1)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        lb.lcs_sweep_incr_fx_noalloc(s, d, h, dev, out, R, arg, stream=stream.cuda_stream)
        stream.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        assert np.array_equal(out.cpu().numpy(), want_v)
        assert (int(R.item()), int(arg.item())) == (want_R, want_arg)
