"""GPU parity of the staged apply kernel (hop source ranges streamed into
shared memory by bulk asynchronous copies; hm_apply_ex flag bit 5 and the
library default) against the CPU oracle, element by element, on shapes that
exercise its edges: blocks smaller than a consumer pass, ragged blocks,
ranges that start off a 16-byte boundary (misaligned vectors, odd hop
offsets), ranges that cross the ends of the vector, many right-hand sides,
H^T, native FP64, and the fallback for plans without a staged form."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [
    ((2,), None),
    ((5, 7), None),
    ((3, 2, 5, 2, 3, 4, 2, 3, 2), None),                       # ragged blocks of the staged split
    ((2,) * 14, None),                                           # binary chain, many high sites
    ((64, 2, 2, 2, 2, 2, 2, 2), ["boson"] + ["spin"] * 7),       # boson as the top site
    ((2, 2, 2, 2, 2, 2, 2, 64), ["spin"] * 7 + ["boson"]),       # spin-boson hops shifted by one element
    ((3, 5, 2, 7, 3, 2, 2, 3), ["spin", "boson", "spin", "boson", "spin", "spin", "spin", "spin"]),
    ((2, 3) * 6, None),                                          # ferrimagnet-like alternation
]


def _status_clean():
    from paper_2606_02169_gb300 import _capi
    assert _capi.device_status(clear=True) == 0, "a bounded wait of the staged kernel gave up"


def _apply(h, x, **kw):
    torch = torch_cuda()
    y = h.apply_ex(x, kernel="staged", **kw)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("dims,kinds", SHAPES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_staged_matches_oracle(dims, kinds, dtype):
    torch = torch_cuda()
    m = W.random_model(list(dims), kinds, nterms=30, seed=21)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 22).astype(dtype).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x)
    h = ham(m)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    got = _apply(h, torch.from_numpy(x).to("cuda", tdt)).double().cpu().numpy()
    check_close(got, ref, abs_bound(m, x), TOL_F64 if dtype == np.float64 else TOL_F32, f"staged {dims}")
    _status_clean()


@pytest.mark.parametrize("nvec", [2, 3, 16])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_staged_many_right_hand_sides(nvec, dtype):
    torch = torch_cuda()
    m = W.random_model([3, 2, 4, 2, 3, 2, 5, 2], None, nterms=30, seed=11)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 12, nvec=nvec).astype(dtype).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x, nvec=nvec)
    h = ham(m)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    got = _apply(h, torch.from_numpy(x).to("cuda", tdt)).double().cpu().numpy()
    check_close(got, ref, abs_bound(m, x), TOL_F64 if dtype == np.float64 else TOL_F32, f"nvec={nvec}")
    _status_clean()


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_staged_unaligned_fp32_vectors(offset):
    """x and y start 4, 8 or 12 bytes past a 16-byte boundary: every staged
    range has an unaligned head and tail copied with plain loads."""
    torch = torch_cuda()
    m = W.random_model([2, 3, 2, 4, 2, 5, 2, 3], None, nterms=26, seed=4)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 5).astype(np.float32).astype(np.float64)
    h = ham(m)
    buf = torch.zeros(D + 4, dtype=torch.float32, device="cuda")
    out = torch.full((D + 4,), float("nan"), dtype=torch.float32, device="cuda")
    buf[offset:offset + D] = torch.from_numpy(x).to("cuda", torch.float32)
    y = h.apply_ex(buf[offset:offset + D], out=out[offset:offset + D], kernel="staged")
    torch.cuda.synchronize()
    ref = oracle.apply(m.sites, m.terms, x)
    check_close(y.double().cpu().numpy(), ref, abs_bound(m, x), TOL_F32, f"offset {offset}")
    o = out.cpu().numpy()
    assert np.isnan(o[:offset]).all() and np.isnan(o[offset + D:]).all(), "staged kernel wrote outside y"
    _status_clean()


def test_staged_transpose_and_native_fp64():
    torch = torch_cuda()
    m = W.random_model([3, 2, 4, 2, 3, 2, 2], None, nterms=30, seed=17, hermitian=False)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 3)
    h = ham(m)
    xt = torch.from_numpy(x).cuda()
    HT = oracle.dense(m.sites, m.terms, sparse=True).T.tocsr()   # the oracle's H, transposed
    refT = HT @ x
    got = _apply(h, xt, transpose=True).cpu().numpy()
    check_close(got, refT, np.asarray(abs(HT) @ np.abs(x)).reshape(-1), TOL_F64, "staged H^T")
    ref = oracle.apply(m.sites, m.terms, x)
    got = _apply(h, xt, native_f64=True).cpu().numpy()
    check_close(got, ref, abs_bound(m, x), 1e-13, "staged native fp64")
    _status_clean()


def test_staged_is_reproducible_on_tavis_cummings():
    torch = torch_cuda()
    m = W.tavis_cummings(8, 64, seed=7)
    h = ham(m)
    x = torch.from_numpy(W.vector(h.D, 8)).cuda()
    a = _apply(h, x).clone()
    b = _apply(h, x)                    # run to run: bit for bit
    assert torch.equal(a, b)
    ref = oracle.apply(m.sites, m.terms, x.cpu().numpy())
    check_close(a.cpu().numpy(), ref, abs_bound(m, x.cpu().numpy()), TOL_F64, "TC N=8")
    _status_clean()


def test_plan_without_staged_form_falls_back():
    """A site of 1500 levels exceeds the staged kernel's block: an explicit
    staged request is refused, hm_apply (the general kernel) runs."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import _capi
    m = W.random_model([3, 1500], ["spin", "boson"], nterms=12, seed=2)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 4)
    h = ham(m)
    xt = torch.from_numpy(x).cuda()
    y = h.apply(xt)
    torch.cuda.synchronize()
    ref = oracle.apply(m.sites, m.terms, x)
    check_close(y.cpu().numpy(), ref, np.full(D, np.abs(ref).max() + 1.0), TOL_F64, "fallback")
    with pytest.raises(_capi.HmError) as ei:
        h.apply_ex(xt, kernel="staged")
    assert ei.value.code == _capi.HM_ERR_UNSUPPORTED
