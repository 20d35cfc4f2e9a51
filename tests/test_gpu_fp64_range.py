"""FP64 storage keeps FP64's exponent range. The default FP64 arithmetic is
a double-float sum on the FP32 pipe; an input element outside its window
(nonzero |x| < 2^-70 or >= 2^71, subnormal, Inf, NaN) is flagged by the split
pass on the device and the same apply then runs in native FP64, and a plan
whose coefficients leave [2^-30, 2^30] runs native FP64 throughout. Checked
element by element against the oracle at the FP64 tolerance on vectors whose
elements span 1e-300 .. 1e+40 within the same rows."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu


def _wide_vector(D, seed, nvec=1):
    """Signed magnitudes 10^u with u drawn from [-300, -40] or [35, 40], mixed
    so that most rows gather from both ranges."""
    rng = np.random.default_rng(seed)
    n = D * nvec
    u = np.where(rng.random(n) < 0.5, rng.uniform(-300, -40, n), rng.uniform(35, 40, n))
    return np.where(rng.random(n) < 0.5, -1.0, 1.0) * 10.0 ** u


SHAPES = [([3, 2, 4, 2, 3], None), ([2, 2, 2, 2, 2, 2, 2, 64], ["spin"] * 7 + ["boson"]), ([2] * 12, None)]


@pytest.mark.parametrize("dims,kinds", SHAPES)
@pytest.mark.parametrize("kernel", [None, "staged", "general"])
def test_wide_range_inputs(dims, kinds, kernel):
    torch = torch_cuda()
    m = W.random_model(dims, kinds, nterms=24, seed=8)
    D = oracle.dimension(m.sites)
    x = _wide_vector(D, 3)
    h = ham(m)
    xt = torch.from_numpy(x).cuda()
    y = h.apply(xt) if kernel is None else h.apply_ex(xt, kernel=kernel)
    torch.cuda.synchronize()
    ref = oracle.apply(m.sites, m.terms, x)
    check_close(y.cpu().numpy(), ref, abs_bound(m, x), TOL_F64, f"wide range {dims} {kernel}")


def test_tiny_rows_alone():
    """Every element near 1e-300: far below float's range, so the whole apply
    runs in native FP64 and matches elementwise."""
    torch = torch_cuda()
    m = W.random_model([2, 3, 2, 4, 2], None, nterms=20, seed=9)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 4) * 1e-300
    h = ham(m)
    y = h.apply(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref = oracle.apply(m.sites, m.terms, x)
    check_close(y.cpu().numpy(), ref, abs_bound(m, x), TOL_F64, "1e-300")
    assert np.abs(ref).max() > 0


def test_coefficient_outside_window():
    torch = torch_cuda()
    m = W.random_model([3, 2, 4, 2, 3], None, nterms=20, seed=10)
    terms = list(m.terms) + [(1, "Sz", -1, "I", 1e-45), (0, "Sp", 2, "Sm", 3e40), (2, "Sp", 0, "Sm", 3e40)]
    m2 = W.Model("tiny_and_huge_coefficients", m.sites, terms, {})
    D = oracle.dimension(m2.sites)
    x = W.vector(D, 5)
    h = ham(m2)
    y = h.apply(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref = oracle.apply(m2.sites, m2.terms, x)
    check_close(y.cpu().numpy(), ref, abs_bound(m2, x), TOL_F64, "coefficients 1e-45 and 3e40")


def test_wide_range_transpose_and_many_rhs():
    torch = torch_cuda()
    m = W.random_model([3, 2, 4, 2, 3], None, nterms=24, seed=12, hermitian=False)
    D = oracle.dimension(m.sites)
    nvec = 3
    x = _wide_vector(D, 6, nvec=nvec)
    h = ham(m)
    y = h.apply(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref = oracle.apply(m.sites, m.terms, x, nvec=nvec)
    check_close(y.cpu().numpy(), ref, abs_bound(m, x), TOL_F64, "wide range nvec=3")
    HT = oracle.dense(m.sites, m.terms, sparse=True).T.tocsr()
    x1 = x.reshape(D, nvec)[:, 0].copy()
    g = h.apply_ex(torch.from_numpy(x1).cuda(), transpose=True, kernel="staged")
    torch.cuda.synchronize()
    check_close(g.cpu().numpy(), HT @ x1, np.asarray(abs(HT) @ np.abs(x1)).reshape(-1), TOL_F64, "wide range H^T")
