"""The Legendre autotuner's process-wide choice cache (host logic of
cr_tune_set / cr_tune_entry; no GPU needed): pinned choices (pairs per
thread and m tile) read back per (grid shape, band limit, precision,
stage), later pins replace earlier ones, and invalid choices are
rejected."""
import pytest

from paper_1308_5299_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    from paper_1308_5299_gb300 import build
    build.build()
    return binding.lib()


def test_pins_read_back_and_replace(lib):
    binding.tune_set(127, 12288, 95, "f64", "adjoint", 8)
    binding.tune_set(127, 12288, 95, "f32", "synthesis", 2, m_tile=2)
    binding.tune_set(127, 12288, 95, "f64", "adjoint", 2)  # replaces the first pin
    rows = [t for t in binding.tune_table() if (t["nring"], t["npix"], t["lmax"]) == (127, 12288, 95)]
    got = {(t["precision"], t["stage"]): (t["pairs_per_thread"], t["m_tile"]) for t in rows}
    assert got == {("f64", "adjoint"): (2, 1), ("f32", "synthesis"): (2, 2)}


def test_sixteen_pairs_only_for_fp32_adjoint(lib):
    binding.tune_set(63, 3072, 47, "f32", "adjoint", 16)
    rows = [t for t in binding.tune_table() if (t["nring"], t["npix"], t["lmax"]) == (63, 3072, 47)]
    assert [t["pairs_per_thread"] for t in rows] == [16]
    with pytest.raises(binding.CRError):
        binding.tune_set(63, 3072, 47, "f32", "synthesis", 16)


@pytest.mark.parametrize("rp,mt,prec,stage", [(3, 1, "f32", "synthesis"), (16, 1, "f64", "adjoint"),
                                               (32, 1, "f32", "adjoint"), (4, 3, "f32", "adjoint"),
                                               (4, 0, "f64", "synthesis"), (1, 2, "bf16", "tc_synthesis")])
def test_invalid_choice_rejected(lib, rp, mt, prec, stage):
    with pytest.raises(binding.CRError) as e:
        binding.tune_set(31, 768, 23, prec, stage, rp, m_tile=mt)
    assert e.value.code == binding.CR_EINVAL
