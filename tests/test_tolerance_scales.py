"""The per-term tolerance scale of sampled-row GPU checks: abs_terms' term
list, applied by the row-wise oracle to |x|, bounds sum_t |c_t| |O_t| |x|
(itself at least the merged (|H| |x|)) row by row, and equals it where every
Sz sits on a spin-1/2 site; its rows agree with its full apply."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import abs_terms, apply_abs_bound, row_abs_bound

MODELS = [W.random_model([3, 2, 4, 2, 3], None, nterms=30, seed=3),
          W.random_model([2, 5, 2, 3], ["spin", "boson", "spin", "spin"], nterms=20, seed=4),
          W.tavis_cummings(5, 8),
          W.ferrimagnet_chain(6),
          W.Model("sy_terms", [("spin", 2), ("spin", 3), ("spin", 2)],
                  [(0, "Sy", 1, "Sx", 0.7), (1, "Sy", -1, "I", -0.4), (0, "Sz", 2, "Sy", 0.5), (2, "Sz", 1, "Sz", 1.2)])]


def _per_term(m, x):
    tot = np.zeros(x.size)
    for t in m.terms:
        tot += abs(oracle.dense(m.sites, [t], sparse=True)) @ np.abs(x)
    return tot


@pytest.mark.parametrize("m", MODELS, ids=[m.name for m in MODELS])
def test_bound_covers_the_per_term_scale(m):
    D = oracle.dimension(m.sites)
    x = W.vector(D, 11)
    rows = np.arange(D)
    b = row_abs_bound(m, x, rows)
    ex = _per_term(m, x)
    merged = abs(oracle.dense(m.sites, m.terms, sparse=True)) @ np.abs(x)
    assert np.all(ex >= merged * (1 - 1e-12))
    assert np.all(b >= ex * (1 - 1e-12))
    if all(not (op == "Sz" and m.sites[s][1] > 2) for (i, oi, j, oj, _) in m.terms for s, op in ((i, oi), (j, oj))
           if s >= 0):
        assert np.allclose(b, ex, rtol=1e-12, atol=0)
    assert np.allclose(apply_abs_bound(m, x), b, rtol=1e-13, atol=0)


def test_abs_terms_replacements():
    m = MODELS[-1]
    t = abs_terms(m)
    assert t[0] == (0, "Sx", 1, "Sx", 0.7)          # |Sy| = Sx elementwise
    assert t[1] == (1, "Sx", -1, "I", 0.4)
    assert t[2] == (0, "I", 2, "Sx", 0.25)         # Sz on spin-1/2 -> (1/2) I
    assert t[3] == (2, "I", 1, "I", 1.2 * 0.5 * 1.0)
