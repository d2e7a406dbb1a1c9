"""The tolerance of the tensor-core tests (1e-2 relative L2) from the
arithmetic: the batched Legendre contraction rounds both operands -- the
generated P~ values and the coefficients -- to BF16 (8-bit significand,
round to nearest even) and accumulates in FP32.  Emulated here with the
oracle's P~ on a small grid, the relative error of F_m(z) = sum_l P~_lm a_lm
is about 2^-9 (about 2e-3): the test tolerance leaves a margin of more than
three, while FP32 accumulation alone is 1e-7."""
import numpy as np

from oracle import geometry, sht
from paper_1308_5299_gb300 import synthetic


def bf16(x):
    """Round FP64 values to BF16 (through FP32, nearest even), back to FP64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_is_nearest_even():
    assert bf16(1.0) == 1.0
    assert bf16(1.0 + 2.0 ** -8) == 1.0  # 1 + 2^-8 is a tie; the even neighbour is 1
    assert bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    rng = np.random.default_rng(0)
    x = rng.normal(size=10000)
    rel = np.abs(bf16(x) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 + 1e-12


def test_bf16_contraction_error_is_a_few_thousandths():
    nside, L = 16, 47
    g = geometry.healpix_grid(nside)
    a = synthetic.random_alm(L, seed=77)
    num = den = 0.0
    for k in range(g["nring"]):
        z = g["z"][k]
        for m in range(L + 1):
            p = sht.plm(L, m, z)
            seg = a[sht.lm_offset(L, m):sht.lm_offset(L, m) + L + 1 - m]
            exact = p @ seg
            rounded = bf16(p) @ (bf16(seg.real) + 1j * bf16(seg.imag))
            num += abs(rounded - exact) ** 2
            den += abs(exact) ** 2
    rel = np.sqrt(num / den)
    assert 5e-4 < rel < 1e-2 / 3, rel
