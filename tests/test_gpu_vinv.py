"""One group factor per lane (hm_apply_ex bit 15): where every factorised
high/low group's low digit has a period dividing the stride between a
lane's elements, the lane forms v once and the member coefficients v*u
once. It rounds differently from the default form, so both are checked
against the oracle; plans whose groups do not allow it run the default
form unchanged."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    (lambda: W.tavis_cummings(8, 64, seed=3), "tc8"),        # boson last: period 64
    (lambda: W.tavis_cummings(10, 16, seed=4), "tc10"),
    (lambda: W.random_model([3, 2, 2, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2], None, nterms=40, seed=5), "mixed"),
    (lambda: W.random_model([5, 2, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 4],
                            [W.BOSON] + [W.SPIN] * 12 + [W.BOSON], nterms=40, seed=6), "bosons"),
]


@pytest.mark.parametrize("make,name", CASES)
@pytest.mark.parametrize("dtype,nvec", [("f64", 1), ("f32", 1), ("f64", 2), ("f32", 4), ("f64", 8)])
def test_group_factor_per_lane_matches_oracle(make, name, dtype, nvec):
    torch = torch_cuda()
    m = make()
    h = ham(m)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    x = torch.from_numpy(W.vector(h.D, 21, nvec=nvec)).to("cuda", tdt)
    xn = x.double().cpu().numpy()
    ref = oracle.apply(m.sites, m.terms, xn, nvec=nvec)
    scale = abs_bound(m, xn)
    tol = TOL_F32 if dtype == "f32" else TOL_F64
    for kw in (dict(), dict(prefetch=True, s=8), dict(s=6, mb=True), dict(s=2), dict(scalar=True)):
        y = h.apply_ex(x, kernel="general", vinv=True, **kw)
        y2 = h.apply_ex(x, kernel="general", vinv=True, **kw)
        torch.cuda.synchronize()
        assert torch.equal(y, y2), f"{name} {kw}: not reproducible"
        check_close(y.double().cpu().numpy(), ref, scale, tol, f"{name} {dtype} nvec={nvec} {kw}")
    yt = h.apply_ex(x, kernel="general", vinv=True, transpose=True)
    Ht = oracle.dense(m.sites, m.terms, sparse=True).T.tocsr()
    reft = np.asarray(Ht @ xn.reshape(h.D, nvec)).reshape(-1)
    scalet = np.asarray(abs(Ht) @ np.abs(xn).reshape(h.D, nvec)).reshape(-1)
    check_close(yt.double().cpu().numpy(), reft, scalet, tol, f"{name} transpose")


def test_group_factor_per_lane_with_split_and_tuning():
    torch = torch_cuda()
    m = W.tavis_cummings(14, 64, seed=7)      # D = 2^20: three spins above the low block
    h = ham(m)
    x = torch.from_numpy(W.vector(h.D, 2)).cuda()
    ref = oracle.apply(m.sites, m.terms, x.cpu().numpy())
    scale = abs_bound(m, x.cpu().numpy())
    y = h.apply_ex(x, kernel="general", vinv=True, split=True, split_sites=2)
    check_close(y.cpu().numpy(), ref, scale, TOL_F64, "vinv + split")
    cfg = h.tune(1, torch.float64)
    check_close(h.apply(x).cpu().numpy(), ref, scale, TOL_F64, f"tuned {cfg}")
