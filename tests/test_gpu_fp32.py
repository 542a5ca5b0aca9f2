"""The float32-storage experiment against the exact fixed-point iterates.

Float32 iterates carry rounding error, so they are compared with a stated
tolerance: after T iterations the offset-normalised values stay within
T * 4e-6 (absolute, in units of the iterate) of the exact ones for the shapes
below; no bound is derived from them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2407_10925_gb300 as lb

    lb.lib()
    return torch, lb


@pytest.mark.parametrize("s,d,h,iters", [(2, 2, 6, 120), (2, 3, 4, 150), (3, 2, 4, 150)])
def test_fp32_tracks_fixed_point(env, orc, s, d, h, iters):
    torch, lb = env
    exact = orc.run(s, d, h, iters, arith="fx")["iterates"][0].astype(np.float64) / 2.0 ** 44
    r = orc.run(s, d, h, 60, arith="fx")["r"] / 2.0 ** 44
    out = torch.empty(s ** (d * h), dtype=torch.float64, device="cuda")
    lb.lcs_fp32_experiment(s, d, h, iters, r, out)
    got = out.cpu().numpy()
    err = np.max(np.abs(got - exact))
    assert err < iters * 4e-6, err
    assert err > 0  # float32 really was used


def test_fp32_rejects_unsupported(env):
    torch, lb = env
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(lb.LcsError):
        lb.lcs_fp32_experiment(4, 2, 1, 3, 0.3, out)
