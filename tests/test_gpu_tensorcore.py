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


import numpy as np
import torch

from gpu_util import rel_l2
from oracle import geometry, sht
from paper_1308_5299_gb300 import synthetic


@pytest.mark.parametrize("nside,lmax,nrhs", [(8, 23, 3), (32, 95, 20), (64, 191, 16)])
def test_tensor_core_batched_synthesis_matches_oracle(nside, lmax, nrhs):
    """Batched synthesis with the Legendre contraction on the tensor cores
    (BF16 operands, FP32 accumulation): every right-hand side within BF16
    accuracy of the FP64 oracle."""
    dev = cuda_device()
    g = geometry.healpix_grid(nside)
    plan = binding.Plan(lmax, nside=nside)
    a = np.stack([synthetic.random_alm(lmax, seed=900 + j) for j in range(nrhs)])
    m = torch.empty((nrhs, g["npix"]), dtype=torch.float32, device=dev)
    plan.sht_synth(torch.from_numpy(a).to(torch.complex64).to(dev), m, tensor_cores=True)
    mh = m.cpu().numpy().astype(np.float64)
    for j in range(nrhs):
        assert rel_l2(mh[j], sht.synth(a[j], lmax, g)) < 1e-2, j


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
        assert rel_l2(mh[sel], ref[sel]) < 1e-2
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
