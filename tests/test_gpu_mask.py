"""Crowded-flavor saturation mask (Sec. 3.1) on the GPU against the oracle.

Integer (byte) output: bit-exact.  Both sides decide saturation on the same
values (the image dtype widened to FP64)."""
import ctypes

import numpy as np
import pytest

from oracle import masking

torch = pytest.importorskip("torch")


def test_rejects_bad_arguments():
    from paper_2109_09334_gb300 import binding as B
    from paper_2109_09334_gb300.build import build
    build()
    lib = B.library()
    fake = 4096  # never dereferenced: every call below is rejected first
    f = lib.sfft_saturation_mask
    assert f(16, 16, B.SFFT_F32, None, fake, 1.0, 1.0, 1, None, fake, None) == B.SFFT_ERR_INVALID
    assert f(16, 16, B.SFFT_F32, fake, fake, 1.0, 1.0, 1, None, None, None) == B.SFFT_ERR_INVALID
    assert f(0, 16, B.SFFT_F32, fake, fake, 1.0, 1.0, 1, None, fake, None) == B.SFFT_ERR_INVALID
    assert f(16, 16, B.SFFT_F32, fake, fake, 1.0, 1.0, 17, None, fake, None) == B.SFFT_ERR_INVALID
    assert f(16, 16, 7, fake, fake, 1.0, 1.0, 1, None, fake, None) == B.SFFT_ERR_INVALID


@pytest.mark.gpu
@pytest.mark.parametrize("n0,n1,grow", [(64, 64, 0), (100, 37, 3), (33, 130, 16), (1, 40, 2), (4096, 4096, 5)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_saturation_mask_matches_oracle(n0, n1, grow, dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import binding as B
    rng = np.random.default_rng(n0 + n1 + grow)
    R = rng.uniform(0, 100, (n0, n1)).astype(dtype)
    S = rng.uniform(0, 100, (n0, n1)).astype(dtype)
    sat_r, sat_s = 99.7, 99.9
    m_in = (rng.random((n0, n1)) > 0.05).astype(np.uint8)
    Rt, St = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
    out = torch.empty((n0, n1), dtype=torch.uint8, device="cuda")
    B.sfft_saturation_mask(Rt, St, sat_r, sat_s, grow, out)
    want = masking.saturation_mask(R.astype(np.float64), S.astype(np.float64), sat_r, sat_s, grow)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    # with an input mask, in place
    mt = torch.from_numpy(m_in).cuda()
    B.sfft_saturation_mask(Rt, St, sat_r, sat_s, grow, mt, d_mask_in=mt)
    torch.cuda.synchronize()
    want2 = masking.saturation_mask(R.astype(np.float64), S.astype(np.float64), sat_r, sat_s, grow, m_in)
    assert np.array_equal(mt.cpu().numpy(), want2)
