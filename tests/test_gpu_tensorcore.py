"""The fifth-generation tensor-core path (tcgen05.mma, BF16 operands, FP32
accumulation in tensor memory): one GEMM tile against the CUDA cores."""
import pytest

from gpu_util import cuda_device
from paper_1308_5299_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [16, 32, 64])
def test_tcgen05_tile_matches_cuda_cores(K):
    cuda_device()
    assert binding.tc_selftest(K) == 0.0


@pytest.mark.parametrize("K", [16, 64])
def test_tcgen05_mn_major_tile(K):
    """The transposed (MN-major) operand layout without swizzle, the one the
    batched adjoint writes: with the K-direction core-matrix stride in the
    descriptor's leading byte offset and the MN-direction stride in its
    stride byte offset the tile reproduces the CUDA-core product exactly;
    the other reading of the two offsets does not."""
    cuda_device()
    e_mn_lead, e_k_lead = binding.tc_selftest_mn(K, 0), binding.tc_selftest_mn(K, 1)
    print("MN-major tile K=%d: max |error| %g (K stride as leading offset), %g (MN stride as leading offset)"
          % (K, e_k_lead, e_mn_lead))
    assert e_k_lead == 0.0 and e_mn_lead > 0.0


import numpy as np
import torch

from gpu_util import rel_l2
from oracle import geometry, sht
from paper_1308_5299_gb300 import synthetic


# BF16 operands: the rounding model of tests/test_bf16_error_model.py gives
# 2.4e-3 relative L2 per transform; hi + lo operands (three MMAs): ~2^-17
# per product, so the FP32 recurrence's ~1e-6 dominates
TOL_BF16 = 5e-3
TOL_SPLIT = 3e-5


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("nside,lmax,nrhs", [(8, 23, 3), (32, 95, 20), (64, 191, 16), (256, 767, 16)])
def test_tensor_core_batched_synthesis_matches_oracle(nside, lmax, nrhs, split):
    """Batched synthesis with the Legendre contraction on the tensor cores
    (BF16 operands, or hi + lo BF16 pairs, FP32 accumulation): every
    right-hand side within the operands' accuracy of the FP64 oracle."""
    dev = cuda_device()
    g = geometry.healpix_grid(nside)
    plan = binding.Plan(lmax, nside=nside, tc_split=split)
    a = np.stack([synthetic.random_alm(lmax, seed=900 + j) for j in range(nrhs)])
    m = torch.empty((nrhs, g["npix"]), dtype=torch.float32, device=dev)
    plan.sht_synth(torch.from_numpy(a).to(torch.complex64).to(dev), m, tensor_cores=True)
    mh = m.cpu().numpy().astype(np.float64)
    errs = [rel_l2(mh[j], sht.synth(a[j], lmax, g)) for j in range(nrhs)]
    print("tensor-core synthesis nside %d lmax %d split %s: max rel L2 %.2e" % (nside, lmax, split, max(errs)))
    tol = TOL_SPLIT if split else TOL_BF16
    for j, e in enumerate(errs):
        assert e < tol, (j, e)


def test_tensor_core_batched_synthesis_full_size_sampled_rings():
    dev = cuda_device()
    nside, lmax, nrhs = 2048, 3000, 16
    g = geometry.healpix_grid(nside)
    plan = binding.Plan(lmax, nside=nside)
    a = np.stack([synthetic.random_alm(lmax, seed=950 + j) for j in range(2)])
    at = torch.zeros((nrhs, sht.n_lm(lmax)), dtype=torch.complex64, device=dev)
    at[0] = torch.from_numpy(a[0]).to(torch.complex64)
    at[nrhs - 1] = torch.from_numpy(a[1]).to(torch.complex64)
    m = torch.empty((nrhs, g["npix"]), dtype=torch.float32, device=dev)
    plan.sht_synth(at, m, tensor_cores=True)
    R = g["nring"]
    rings = np.array([0, 5, nside - 1, nside, 2 * nside - 1, R - 1])
    for j, jj in [(0, 0), (1, nrhs - 1)]:
        ref = sht.synth(a[j], lmax, g, rings=rings)
        mh = m[jj].cpu().numpy().astype(np.float64)
        sel = np.concatenate([np.arange(g["off"][k], g["off"][k] + g["nphi"][k]) for k in rings])
        assert rel_l2(mh[sel], ref[sel]) < TOL_BF16
    # throughput: 16 right-hand sides on the tensor cores vs 16 FP32 syntheses
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    plan.sht_synth(at, m, tensor_cores=True)
    e1.record()
    for j in range(nrhs):
        plan.sht_synth(at[j], m[j])
    e2.record()
    torch.cuda.synchronize()
    print("tensor-core 16-RHS synthesis %.1f ms, 16 FP32 syntheses %.1f ms" % (e0.elapsed_time(e1), e1.elapsed_time(e2)))


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("nside,lmax,nrhs", [(8, 23, 3), (32, 95, 20), (64, 191, 16), (256, 767, 16)])
def test_tensor_core_batched_adjoint_matches_oracle(nside, lmax, nrhs, split):
    """Batched adjoint synthesis with the Legendre contraction on the tensor
    cores (BF16 operands, or hi + lo BF16 pairs): every right-hand side
    within the operands' accuracy of the FP64 oracle (Y^T, no quadrature
    weights), Im(a_l0) exactly zero."""
    dev = cuda_device()
    g = geometry.healpix_grid(nside)
    plan = binding.Plan(lmax, nside=nside, tc_split=split)
    maps = np.stack([synthetic.random_map(g["npix"], seed=700 + j) for j in range(nrhs)])
    out = torch.empty((nrhs, sht.n_lm(lmax)), dtype=torch.complex64, device=dev)
    plan.sht_adjoint(torch.from_numpy(maps).to(torch.float32).to(dev), out, tensor_cores=True)
    oh = out.cpu().numpy().astype(np.complex128)
    l, m = sht.lm_arrays(lmax)
    assert np.all(oh[:, m == 0].imag == 0)
    errs = [rel_l2(oh[j], sht.adjoint(maps[j], lmax, g)) for j in range(nrhs)]
    print("tensor-core adjoint nside %d lmax %d split %s: max rel L2 %.2e" % (nside, lmax, split, max(errs)))
    tol = TOL_SPLIT if split else TOL_BF16
    for j, e in enumerate(errs):
        assert e < tol, (j, e)


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("name,nrhs", [("nside32_lmax95", 18), ("nside16_lmax47", 5)])
def test_tensor_core_batched_apply_A_matches_oracle(name, nrhs, split):
    """A = S^-1 + B Y^T N^-1 Y B for many right-hand sides with both Legendre
    stages on the tensor cores, against the FP64 oracle operator."""
    from oracle import operators

    dev = cuda_device()
    cfg, cl, bl, ninv = synthetic.problem_inputs(name)
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    plan = binding.Plan(cfg["lmax"], nside=cfg["nside"], cl=cl, bl=bl, ninv=torch.from_numpy(ninv).to(dev),
                        tc_split=split)
    xs = np.stack([prob.clean(synthetic.draw_prior(cl, index=40 + j)) for j in range(nrhs)])
    y = torch.empty((nrhs, sht.n_lm(cfg["lmax"])), dtype=torch.complex64, device=dev)
    plan.apply_A(torch.from_numpy(xs).to(torch.complex64).to(dev), y, tensor_cores=True)
    yh = y.cpu().numpy().astype(np.complex128)
    errs = [rel_l2(yh[j], operators.apply_A(prob, xs[j])) for j in range(nrhs)]
    print("tensor-core apply_A %s split %s: max rel L2 %.2e" % (name, split, max(errs)))
    tol = TOL_SPLIT if split else TOL_BF16
    for j, e in enumerate(errs):
        assert e < tol, (j, e)


def test_tensor_core_batched_adjoint_full_size_sampled_rings():
    """Nside 2048, lmax 3000, 16 right-hand sides: maps that are non-zero on
    a few rings (pole, cap edge, equator), so the oracle's adjoint restricted
    to those rings is the exact answer; slots 0 and 15 carry data."""
    dev = cuda_device()
    nside, lmax, nrhs = 2048, 3000, 16
    g = geometry.healpix_grid(nside)
    plan = binding.Plan(lmax, nside=nside)
    R = g["nring"]
    rings = np.array([0, 5, nside - 1, nside, 2 * nside - 1, R - 1])
    sel = np.concatenate([np.arange(g["off"][k], g["off"][k] + g["nphi"][k]) for k in rings])
    maps = np.zeros((2, g["npix"]))
    for j in range(2):
        maps[j, sel] = synthetic.random_map(g["npix"], seed=960 + j)[sel]
    mt = torch.zeros((nrhs, g["npix"]), dtype=torch.float32, device=dev)
    mt[0] = torch.from_numpy(maps[0]).to(torch.float32)
    mt[nrhs - 1] = torch.from_numpy(maps[1]).to(torch.float32)
    out = torch.empty((nrhs, sht.n_lm(lmax)), dtype=torch.complex64, device=dev)
    plan.sht_adjoint(mt, out, tensor_cores=True)
    for j, jj in [(0, 0), (1, nrhs - 1)]:
        ref = sht.adjoint(maps[j], lmax, g, rings=rings)
        assert rel_l2(out[jj].cpu().numpy().astype(np.complex128), ref) < TOL_BF16
    assert float(out[1:nrhs - 1].abs().max()) == 0.0
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    plan.sht_adjoint(mt, out, tensor_cores=True)
    e1.record()
    for j in range(nrhs):
        plan.sht_adjoint(mt[j], out[j])
    e2.record()
    torch.cuda.synchronize()
    print("tensor-core 16-RHS adjoint %.1f ms, 16 FP32 adjoints %.1f ms" % (e0.elapsed_time(e1), e1.elapsed_time(e2)))
