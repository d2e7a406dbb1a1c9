"""Differentiation through the CUDA solve (torch.autograd over the C ABI):
gradients of a constrained realization and of the Wiener-filter data term
with respect to C_l and the N^-1 map, against the dense oracle gradient at
Nside 8 and against central finite differences (relative step 1e-4) of the
GPU path itself at Nside 512 / lmax 1023 with an 8-RHS batch."""
import numpy as np
import pytest
import torch

from gpu_util import cuda_device, rel_l2
from oracle import geometry, gradients, operators, sht
from paper_1308_5299_gb300 import autodiff, binding, synthetic

pytestmark = pytest.mark.gpu


def loss_of(x, w):
    """L = <w, x> per right-hand side, summed (real inner product)."""
    L = int(round((np.sqrt(8 * w.shape[-1] + 1) - 3) / 2))
    m = np.concatenate([np.full(L + 1 - mm, mm) for mm in range(L + 1)])
    wt = torch.from_numpy(np.where(m == 0, 1.0, 2.0)).to(x.device)
    return (wt * (w.real * x.real + w.imag * x.imag)).sum()


def test_realization_gradient_matches_dense_oracle():
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside8_lmax23")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    rng = np.random.default_rng(21)
    d = rng.normal(size=g["npix"]) * 20.0
    w = prob.clean(rng.normal(size=sht.n_lm(prob.lmax)) + 1j * rng.normal(size=sht.n_lm(prob.lmax)))
    seed = 99
    gcl_ref, gn_ref, x_ref = gradients.realization_grad(prob, seed, d, w)
    tcl = torch.tensor(cl, dtype=torch.float64, requires_grad=True)
    tn = torch.tensor(ninv, dtype=torch.float64, device=dev, requires_grad=True)
    x = autodiff.realization(tcl, tn, bl, cfg["nside"], d=torch.from_numpy(d[None]).to(dev), seed=seed)
    assert rel_l2(x[0].detach().cpu().numpy(), x_ref) < 1e-9
    loss_of(x[0], torch.from_numpy(w).to(dev)).backward()
    assert rel_l2(tcl.grad.numpy(), gcl_ref) < 1e-8
    assert rel_l2(tn.grad.cpu().numpy(), gn_ref) < 1e-8


def test_wf_data_term_gradient_matches_dense_oracle():
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside8_lmax23")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    d = np.random.default_rng(22).normal(size=g["npix"]) * 20.0
    D_ref, gcl_ref, gn_ref, _ = gradients.wf_data_term(prob, d)
    tcl = torch.tensor(cl, dtype=torch.float64, requires_grad=True)
    tn = torch.tensor(ninv, dtype=torch.float64, device=dev, requires_grad=True)
    D = autodiff.wf_data_term(tcl, tn, bl, cfg["nside"], torch.from_numpy(d).to(dev))
    assert abs(float(D.detach()) - D_ref) < 1e-9 * abs(D_ref)
    D.backward()
    assert rel_l2(tcl.grad.numpy(), gcl_ref) < 1e-8
    assert rel_l2(tn.grad.cpu().numpy(), gn_ref) < 1e-8


def test_realization_gradient_finite_differences_nside512():
    """Directional central differences along random relative perturbations
    of C_l and of N^-1 (step 1e-4) against <grad, direction>."""
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside512_lmax1023")
    nside, nrhs, seed = cfg["nside"], 8, 5
    rng = np.random.default_rng(23)
    w = torch.from_numpy(rng.normal(size=(nrhs, sht.n_lm(cfg["lmax"]))) * 1.0 + 0j).to(dev)
    tn0 = torch.tensor(ninv, dtype=torch.float64, device=dev)

    def loss(c, n):
        with torch.no_grad():
            x = autodiff.realization(torch.tensor(c), n, bl, nside, seed=seed, nrhs=nrhs)
            return float(loss_of(x, w))

    tcl = torch.tensor(cl, dtype=torch.float64, requires_grad=True)
    tn = tn0.clone().requires_grad_(True)
    x = autodiff.realization(tcl, tn, bl, nside, seed=seed, nrhs=nrhs)
    loss_of(x, w).backward()
    h = 1e-4
    dc = cl * rng.choice([-1.0, 1.0], size=cl.shape)
    fd = (loss(cl + h * dc, tn0) - loss(cl - h * dc, tn0)) / (2 * h)
    an = float((tcl.grad.numpy() * dc).sum())
    assert abs(fd - an) < 1e-5 * max(abs(an), 1e-30), (fd, an)
    dn = tn0 * torch.from_numpy(rng.choice([-1.0, 1.0], size=ninv.shape)).to(dev)
    fd = (loss(cl, tn0 + h * dn) - loss(cl, tn0 - h * dn)) / (2 * h)
    an = float((tn.grad * dn).sum())
    assert abs(fd - an) < 1e-5 * max(abs(an), 1e-30), (fd, an)


def test_wf_loglike_gradient_with_hutchinson_matches_oracle():
    """Whole Wiener-filter log-likelihood gradient: the data term exactly and
    the log-determinant term by Hutchinson with the same Philox probes on
    both sides, against the dense oracle."""
    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside8_lmax23")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    d = np.random.default_rng(24).normal(size=g["npix"]) * 20.0
    seed, K = 31, 6
    D_ref, gcl_d, gn_d, _ = gradients.wf_data_term(prob, d)
    gcl_h, gn_h = gradients.logdet_grad_hutchinson(prob, seed, K)
    D, gcl, gn = autodiff.wf_loglike_grad(torch.tensor(cl), torch.tensor(ninv, device=dev), bl, cfg["nside"],
                                          torch.from_numpy(d).to(dev), nprobe=K, seed=seed)
    assert abs(D - D_ref) < 1e-9 * abs(D_ref)
    assert rel_l2(gcl.cpu().numpy(), gcl_d + gcl_h) < 1e-8
    assert rel_l2(gn.cpu().numpy(), gn_d + gn_h) < 1e-8
