"""Batched realizations captured into one CUDA graph (cr_batch_*): several
right-hand sides on two plans of different resolution; the graph replay
reproduces the uncaptured fixed-count CR-Solves exactly, and every
realization converges to its exact answer x_true of b = A x_true."""
import numpy as np
import pytest
import torch

from gpu_util import cuda_device
from oracle import geometry, sht
from paper_1308_5299_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


def make_plan(nside, lmax, fwhm, stream, dev):
    cl = synthetic.cl_spectrum(lmax, True, "c2")
    bl = synthetic.gaussian_beam(lmax, fwhm)
    ninv = synthetic.mask(nside, 10.0, 20, 4.0 * 3438.0 / nside) / synthetic.noise_rms(nside, 10.0, 60.0) ** 2
    plan = binding.Plan(lmax, nside=nside, cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev), levels="default",
                        stream=stream)
    return plan, cl


def test_batch_graph_matches_direct_solves():
    dev = cuda_device()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        _run(dev, stream)


def _run(dev, stream):
    specs = [(64, 191, 120.0, 3), (32, 95, 240.0, 2)]
    plans, xs, bs, xts = [], [], [], []
    for k, (nside, lmax, fwhm, nr) in enumerate(specs):
        plan, cl = make_plan(nside, lmax, fwhm, stream, dev)
        xt = torch.from_numpy(np.stack([synthetic.draw_prior(cl, index=50 + 10 * k + j) for j in range(nr)])).to(dev)
        b = torch.empty_like(xt)
        plan.apply_A(xt, b)
        plans.append(plan)
        bs.append(b)
        xs.append(torch.zeros_like(b))
        xts.append(xt)
    cycles, mode = 8, binding.CR_MIXED
    refs = []
    for plan, b in zip(plans, bs):
        r = torch.empty_like(b)
        plan.solve(b, r, eps=0.0, max_cycles=cycles, mode=mode | binding.CR_FIXED, check=False)
        refs.append(r)
    batch = binding.Batch(plans, xs, bs, cycles, mode)
    assert batch.nodes() > 100
    for x in xs:
        x.zero_()
    batch.run()
    torch.cuda.synchronize()
    for plan, x, r, xt, (nside, lmax, _, nr) in zip(plans, xs, refs, xts, specs):
        assert torch.equal(x, r)
        for j in range(nr):
            m = torch.empty(12 * nside * nside, dtype=torch.float64, device=dev)
            plan.sht_synth(x[j] - xt[j], m)
            assert float(m.abs().max()) < 1e-3
    # a second replay on new right-hand sides bound at the same addresses
    bs[0].mul_(2.0)
    batch.run()
    torch.cuda.synchronize()
    assert torch.allclose(xs[0], 2.0 * refs[0], rtol=1e-9, atol=0)
    batch.close()
