"""Failures the library detects and reports as status codes, injected from
the host (no GPU fault, trap or hang):
- an inverse-noise map with a NaN or a negative weight is refused when the
  plan is created;
- smoother blocks forced non-SPD -- an explicit zero ridge on the Nside 32
  problem, whose assembled block matrix is indefinite on every level --
  report the incomplete-Cholesky breakdown;
- a corrupted factor in a checkpoint is refused by its checksum (in
  test_gpu_precompute)."""
import numpy as np
import pytest
import torch

from gpu_util import cuda_device
from oracle import multilevel
from paper_1308_5299_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bad", [float("nan"), -1.0, float("inf")])
def test_bad_inverse_noise_refused(bad):
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside16_lmax47")
    ninv = ninv.copy()
    ninv[123] = bad
    with pytest.raises(binding.CRError) as e:
        binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev))
    assert e.value.code == binding.CR_EINVAL
    assert "pixel 123" in str(e.value)


def test_zero_ridge_reports_icc_breakdown():
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside32_lmax95")
    t = multilevel.level_table(cfg["nside"], cfg["lmax"])
    levels = [dict(nside_h=l["nside_h"], lmax_h=l["lmax_h"], n_rec=l["n_rec"], fl=l["fl"]) for l in t["levels"]]
    with pytest.raises(binding.CRError) as e:
        binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                     levels=levels, lmax_dense=t["bottom"]["lmax_h"], ridge_alpha=[0.0] * len(levels))
    assert e.value.code == binding.CR_EICC
