"""Host-side part of the convergence diagnostics: the per-l norm of the real
field's l component, against the explicit sum over (l, m) built from the
oracle's index arrays, and the identity ||a||^2 = sum_l norm_l^2 = <a, a>."""
import numpy as np

from oracle import sht
from paper_1308_5299_gb300 import diagnostics, synthetic


def test_per_l_norm_matches_explicit_sum():
    L = 37
    a = synthetic.random_alm(L, seed=12)
    l, m = sht.lm_arrays(L)
    ref = np.zeros(L + 1)
    np.add.at(ref, l, np.where(m == 0, 1.0, 2.0) * np.abs(a) ** 2)
    np.testing.assert_allclose(diagnostics.per_l_norm(a, L), np.sqrt(ref), rtol=1e-13)
    # total: the real-basis inner product <a, a>
    dot = np.sum(np.where(m == 0, 1.0, 2.0) * np.abs(a) ** 2)
    np.testing.assert_allclose(np.sum(diagnostics.per_l_norm(a, L) ** 2), dot, rtol=1e-13)
