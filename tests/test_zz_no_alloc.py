"""The allocation-free synthesis entry point (cr_sht_synth_noalloc), for
callers that cannot allocate device memory and so cannot create a plan.

Called through the C ABI and compared with the plan-based cr_sht_synth on
the same inputs, within the FP64 transform tolerance of the parity tests,
on two calls in a row (the static scratch is shared and keeps the previous
call's contents).  Collected last so that a stop-at-first-failure run has
run every other test first; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import cuda_device, rel_l2
from paper_1308_5299_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def dev():
    return cuda_device()


# (1, 16384): the largest accepted band limit, where the seed's log-product
# runs over the most terms (the equator ring's P~_mm does not underflow there)
@pytest.mark.parametrize("nside,lmax", [(64, 191), (256, 767), (1, 16384)])
def test_noalloc_matches_plan_synthesis(dev, nside, lmax):
    plan = binding.Plan(lmax, nside=nside)
    npix = 12 * nside * nside
    for call, seed in enumerate((41, 42)):  # two calls in a row, different inputs
        a = torch.from_numpy(synthetic.random_alm(lmax, seed=seed)).to(dev)
        ref = torch.empty(npix, dtype=torch.float64, device=dev)
        plan.sht_synth(a, ref)
        out = torch.full((npix,), np.nan, dtype=torch.float64, device=dev)
        binding.sht_synth_noalloc(nside, lmax, a, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < TOL64, (call, nside, lmax)


def test_noalloc_rejects_lmax_beyond_plan_range(dev):
    lib = binding.lib()
    a = torch.zeros(16, dtype=torch.complex128, device=dev)
    m = torch.zeros(12, dtype=torch.float64, device=dev)
    rc = lib.cr_sht_synth_noalloc(1, 16385, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(m.data_ptr()), None)
    assert rc == -1  # CR_EINVAL before any buffer is touched
    assert b"16384" in lib.cr_last_error()


def test_noalloc_rejects_sizes_beyond_scratch(dev):
    lib = binding.lib()
    a = torch.zeros(binding.n_lm(2047), dtype=torch.complex128, device=dev)
    m = torch.zeros(12 * 512 * 512, dtype=torch.float64, device=dev)
    rc = lib.cr_sht_synth_noalloc(512, 2047, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(m.data_ptr()), None)
    assert rc == -1  # CR_EINVAL: (4*512-1)*2048*16 bytes > 16 MiB
    assert b"16 MiB" in lib.cr_last_error()
