"""The allocation-free spectral upsampling entry point (psfd_spectral_upsample_static).

It serves callers that cannot allocate device memory during a call; its scratch
is a fixed array inside the library.  Checked against the allocating entry point
(psfd_spectral_upsample) through the C ABI, on two calls in a row with different
data (the second call reuses the scratch the first one left behind).  This file
is collected last on purpose.
"""
import pytest
import torch

from paper_2607_25330_b300 import inputs as I
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def test_static_upsample_matches_the_allocating_one_on_consecutive_calls():
    from paper_2607_25330_b300 import psfd
    cases = [((2, 3, 16, 32, 32), (32, 64, 64), 3), ((1, 3, 32, 16, 64), (64, 16, 128), 4)]
    for shape, (nz, ny, nx), seed in cases:
        src = torch.from_numpy(I.random_field(shape, seed)).to(torch.complex64).cuda()
        ref = psfd.spectral_upsample(src, nz, ny, nx)
        out = psfd.spectral_upsample_static(src, nz, ny, nx)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu(), ref.cpu()) < 1e-6


def test_static_upsample_rejects_requests_beyond_its_scratch():
    from paper_2607_25330_b300 import psfd
    src = torch.zeros((5, 3, 32, 128, 128), dtype=torch.complex64, device="cuda")   # 7.9M entries > 2^21
    with pytest.raises(psfd.PsfdError) as e:
        psfd.spectral_upsample_static(src, 32, 128, 128)
    assert e.value.code == psfd.PSFD_ERR_ARG
