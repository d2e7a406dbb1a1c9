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
