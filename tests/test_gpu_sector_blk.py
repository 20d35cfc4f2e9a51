"""Block form of the sector apply (prefix blocks of contiguous packed states,
per-suffix tables) against the sector oracle and against the per-row kernel
(hm_apply_ex flag bit 4 on a sector plan), on systems large enough to have
prefix sites: all-to-all couplings (prefix-only, coupled and suffix-only
channels of every kind), bosons on either side of the split, several
right-hand sides and both storage types."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, check_close, torch_cuda
from test_gpu_sector import _abs_scale, _chain, _conserving, _ham

pytestmark = pytest.mark.gpu

CASES = [
    ((2,) * 15, ("spin",) * 15, 7),                          # 1 prefix site
    ((2,) * 16, ("spin",) * 16, 8),                          # 2 prefix sites
    ((6,) + (2,) * 12, ("boson",) + ("spin",) * 12, 6),      # boson prefix
    ((3, 2) + (2,) * 10 + (5,), ("spin",) * 12 + ("boson",), 7),  # boson in the suffix
]


@pytest.mark.parametrize("dims,kinds,K", CASES)
@pytest.mark.parametrize("dtype,nvec", [(np.float64, 1), (np.float32, 1), (np.float64, 3)])
def test_block_form_matches_oracle_and_rows(dims, kinds, K, dtype, nvec):
    torch = torch_cuda()
    sites, terms = _conserving(dims, kinds, 11)
    h = _ham(sites, terms, K)
    n = oracle.sector_dimension(sites, K)
    assert h.D == n
    x = W.vector(n, 40 + K, nvec=nvec)
    if dtype == np.float32:
        x = x.astype(np.float32).astype(np.float64)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    xt = torch.from_numpy(x).to("cuda", tdt)
    y = h.apply(xt)
    yr = h.apply_ex(xt, kernel="rows")
    y2 = h.apply(xt)
    torch.cuda.synchronize()
    assert torch.equal(y, y2), "block form not reproducible"
    ref = oracle.sector_apply(sites, terms, K, x, nvec=nvec)
    scale = _abs_scale(sites, terms, K, x, nvec)
    tol = TOL_F64 if dtype == np.float64 else TOL_F32
    check_close(y.double().cpu().numpy(), ref, scale, tol, f"block {dims} K={K}")
    check_close(yr.double().cpu().numpy(), ref, scale, tol, f"rows {dims} K={K}")


@pytest.mark.parametrize("K", [0, 1, 10, 19, 20])
def test_block_form_ring_edge_sectors(K):
    """Periodic chain of 20 spin-1/2 (the closing bond couples the first
    prefix site with the last suffix site), extreme and middle sectors."""
    torch = torch_cuda()
    sites, terms = _chain(20, 2, seed=3)
    h = _ham(sites, terms, K)
    x = W.vector(h.D, 7 + K)
    y = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.sector_apply(sites, terms, K, x)
    check_close(y, ref, _abs_scale(sites, terms, K, x), TOL_F64, f"ring K={K}")
