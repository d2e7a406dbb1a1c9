"""Parity of the CUDA diagonal-preconditioned CG comparator (the method the
paper compares against, Sections 1 and 2.4) with the oracle's CG: same
preconditioner (inverse of 1/C_l + b_l^2 times the Delta m = 0 ring-formula
diagonal of Y^T N^-1 Y), same iterates, and convergence to the exact answer
x_true of b = A x_true."""
import numpy as np
import pytest
import torch

from gpu_util import cuda_device, rel_l2
from oracle import geometry, operators, sht, solvers
from paper_1308_5299_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside32_lmax95")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev))
    l = prob.l
    with np.errstate(divide="ignore"):
        sinv = np.where(prob.active, 1.0 / np.where(prob.active, cl[l], 1.0), 0.0)
    diag = sinv + bl[l] ** 2 * operators.diag_inv_noise_dm0(prob)
    pc = np.where(prob.active & (diag > 0), 1.0 / np.where(diag > 0, diag, 1.0), 0.0)
    return dict(dev=dev, prob=prob, plan=plan, pc=pc, cl=cl)


@pytest.mark.parametrize("k", [1, 5, 12])
def test_cg_iterates_match_oracle(case, k):
    prob, plan, dev = case["prob"], case["plan"], case["dev"]
    b = operators.apply_A(prob, prob.clean(synthetic.draw_prior(case["cl"], index=11)))
    xs = []
    solvers.pcg(lambda v: operators.apply_A(prob, v), b, case["pc"], prob.lmax, tol=0.0, maxiter=k,
                callback=lambda it, x, rel: xs.append(x.copy()))
    x = torch.empty(sht.n_lm(prob.lmax), dtype=torch.complex128, device=dev)
    cyc, rel, hist, rc = plan.solve(torch.from_numpy(b).to(dev), x, eps=0.0, max_cycles=k,
                                    mode=binding.CR_F64 | binding.CR_CG, check=False)
    assert cyc[0] == k
    assert rel_l2(x.cpu().numpy(), xs[-1]) < 1e-9


def test_cg_converges_to_exact_answer(case):
    prob, plan, dev = case["prob"], case["plan"], case["dev"]
    x_true = prob.clean(synthetic.draw_prior(case["cl"], index=12))
    b = operators.apply_A(prob, x_true)
    x = torch.empty(sht.n_lm(prob.lmax), dtype=torch.complex128, device=dev)
    cyc, rel, hist = plan.solve(torch.from_numpy(b).to(dev), x, eps=1e-22, max_cycles=20000,
                                mode=binding.CR_F64 | binding.CR_CG)
    assert rel[0] < 1e-11
    err = sht.synth(x.cpu().numpy() - x_true, prob.lmax, prob.grid)
    assert np.max(np.abs(err)) < 1e-3
