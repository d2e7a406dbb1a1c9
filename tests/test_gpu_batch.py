"""Batched realizations captured into one CUDA graph (cr_batch_*): several
right-hand sides on two plans of different resolution; the graph replay
reproduces the uncaptured fixed-count CR-Solves exactly, and every
realization converges to its exact answer x_true of b = A x_true."""
import numpy as np
import pytest
import torch

from gpu_util import cuda_device
from oracle import sht
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


@pytest.mark.parametrize("top_f32", [False, True])
def test_tensor_core_cycles_converge_to_exact_answers(top_f32):
    """CR_MIXED | CR_TC_CYCLES: 18 right-hand sides (a group of 16 and one of
    2) whose FP32 cycles run together with every Legendre stage on the
    tensor cores; the FP64 outer residual drives each to its exact answer
    x_true of b = A x_true, and the residual history shrinks at a rate close
    to the per-right-hand-side FP32 cycles."""
    dev = cuda_device()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        plan, cl = make_plan(64, 191, 120.0, stream, dev)
        nr = 18
        xt = torch.from_numpy(np.stack([synthetic.draw_prior(cl, index=200 + j) for j in range(nr)])).to(dev)
        b = torch.empty_like(xt)
        plan.apply_A(xt, b)
        x = torch.zeros_like(b)
        mode = binding.CR_MIXED | binding.CR_TC_CYCLES | (binding.CR_TC_TOP_F32 if top_f32 else 0)
        cyc, rel, hist = plan.solve(b, x, eps=1e-20, max_cycles=40, mode=mode)
        assert all(c <= 40 for c in cyc) and max(rel) < 1e-10
        for j in range(nr):
            m = torch.empty(12 * 64 * 64, dtype=torch.float64, device=dev)
            plan.sht_synth(x[j] - xt[j], m)
            assert float(m.abs().max()) < 1e-4
        # convergence per cycle against the per-right-hand-side FP32 cycles
        xr = torch.zeros_like(b[0])
        _, _, href = plan.solve(b[0], xr, eps=0.0, max_cycles=4, mode=binding.CR_MIXED | binding.CR_FIXED,
                                check=False)[:3]
        h_tc = hist[0][:3]
        assert h_tc[2] < 3.0 * href[0][2] + 1e-12, (h_tc, href[0][:3])


@pytest.mark.parametrize("top_f32", [False, True])
def test_tensor_core_cycles_in_a_graph_match_direct(top_f32):
    dev = cuda_device()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        specs = [(64, 191, 120.0, 17), (32, 95, 240.0, 3)]
        plans, xs, bs, refs = [], [], [], []
        cycles, mode = 3, binding.CR_MIXED | binding.CR_TC_CYCLES | (binding.CR_TC_TOP_F32 if top_f32 else 0)
        for k, (nside, lmax, fwhm, nr) in enumerate(specs):
            plan, cl = make_plan(nside, lmax, fwhm, stream, dev)
            xt = torch.from_numpy(np.stack([synthetic.draw_prior(cl, index=300 + 20 * k + j)
                                            for j in range(nr)])).to(dev)
            b = torch.empty_like(xt)
            plan.apply_A(xt, b)
            r = torch.zeros_like(b)
            plan.solve(b, r, eps=0.0, max_cycles=cycles, mode=mode | binding.CR_FIXED, check=False)
            plans.append(plan)
            bs.append(b)
            xs.append(torch.zeros_like(b))
            refs.append(r)
        batch = binding.Batch(plans, xs, bs, cycles, mode)
        for x in xs:
            x.zero_()
        batch.run()
        torch.cuda.synchronize()
        for x, r in zip(xs, refs):
            assert torch.equal(x, r)
        batch.close()


@pytest.mark.parametrize("mode,cycles", [(binding.CR_MIXED, 3),
                                         (binding.CR_MIXED | binding.CR_TC_CYCLES | binding.CR_TC_SPLIT, 3),
                                         (binding.CR_MIXED | binding.CR_TC_CYCLES, 6)])
def test_batch_graph_at_the_mixed_resolution_sizes(mode, cycles):
    """The batch of the benchmark's mixed-resolution measurement at its sizes
    (Nside 1024 / lmax 2047 and Nside 512 / lmax 1023, the first two of its
    realizations each, the cycle counts it reports for the FP32 cycles, the
    split tensor-core cycles and the plain-BF16 ones): the graph replay
    equals the uncaptured solves and every realization is within 1 uK
    max-pixel of its exact answer x_true of b = A x_true."""
    dev = cuda_device()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        plans, xs, bs, xts, refs, npx = [], [], [], [], [], []
        for k, name in enumerate(["nside1024_lmax2047", "nside512_lmax1023"]):
            cfg, cl, bl, ninv = synthetic.problem_inputs(name)
            plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                                stream=stream, levels="default")
            xt = torch.from_numpy(np.stack([synthetic.draw_prior(cl, index=100 * (k + 1) + j)
                                            for j in range(2)])).to(dev)
            b = torch.empty_like(xt)
            plan.apply_A(xt, b)
            r = torch.zeros_like(b)
            plan.solve(b, r, eps=0.0, max_cycles=cycles, mode=mode | binding.CR_FIXED, check=False)
            plans.append(plan)
            xs.append(torch.zeros_like(b))
            bs.append(b)
            xts.append(xt)
            refs.append(r)
            npx.append(12 * cfg["nside"] ** 2)
        batch = binding.Batch(plans, xs, bs, cycles, mode)
        batch.run()
        torch.cuda.synchronize()
        for plan, x, r, xt, n in zip(plans, xs, refs, xts, npx):
            assert torch.equal(x, r)
            for j in range(x.shape[0]):
                m = torch.empty(n, dtype=torch.float64, device=dev)
                plan.sht_synth(x[j] - xt[j], m)
                assert float(m.abs().max()) < 1.0
        batch.close()
