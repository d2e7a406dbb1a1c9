"""Parity of the CUDA right-hand-side generator cr_draw (Section 2.3: the
Wiener-filter term B Y^T N^-1 d plus the constrained-realization
fluctuation terms) with the oracle's independent Philox4x32-10 and direct
adjoint SHT, for several right-hand sides, with and without data and
fluctuations, at C_0 = C_1 = 0 and at the wide monopole prior."""
import numpy as np
import pytest
import torch

from gpu_util import cuda_device, rel_l2
from oracle import draw, geometry, operators, sht
from paper_1308_5299_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["nside32_lmax95", "nside8_lmax23"])
@pytest.mark.parametrize("fluct,with_d", [(True, False), (True, True), (False, True)])
def test_draw_matches_oracle(name, fluct, with_d):
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs(name)
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev))
    nrhs = 3
    d = np.stack([synthetic.random_map(g["npix"], seed=40 + j) * 30.0 for j in range(nrhs)]) if with_d else None
    b = torch.empty((nrhs, sht.n_lm(prob.lmax)), dtype=torch.complex128, device=dev)
    seed = 0x1234_5678_9ABC_DEF0
    plan.draw(seed, b, d=None if d is None else torch.from_numpy(d).to(dev), fluct=fluct)
    for j in range(nrhs):
        ref = draw.draw_rhs(prob, seed, None if d is None else d[j], fluct=fluct, rhs=j)
        assert rel_l2(b[j].cpu().numpy(), ref) < 1e-12, j
