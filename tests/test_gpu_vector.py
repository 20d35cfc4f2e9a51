"""Several right-hand sides per lane: with nvec a multiple of 4 (FP32) or 2
(FP32, FP64 double-float) and aligned vectors, the general kernel handles
that many consecutive right-hand sides of one state per lane. Each right-hand
side takes the same operations in the same order as with one per lane, so
the results are bit-identical to the scalar form (flag bit 13), and both
match the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [
    ((2, 3, 2, 3, 2, 3, 2, 3), None),          # ragged low block, spin-1/2 and spin-1
    ((3, 3, 3, 3, 3, 3, 3), None),             # spin-1 chain
    ((2, 2, 2, 2, 2, 2, 9), [W.SPIN] * 6 + [W.BOSON]),   # boson last
    ((7, 2, 2, 2, 2, 2, 2), [W.BOSON] + [W.SPIN] * 6),   # boson first (a high site)
]


def _model(dims, kinds, seed):
    return W.random_model(list(dims), kinds, nterms=30, seed=seed)


@pytest.mark.parametrize("dims,kinds", SHAPES)
@pytest.mark.parametrize("dtype,nvec", [("f32", 2), ("f32", 4), ("f32", 8), ("f32", 12), ("f32", 16),
                                        ("f32", 6), ("f64", 2), ("f64", 4), ("f64", 6)])
def test_vector_lanes_bit_identical_to_scalar_and_match_oracle(dims, kinds, dtype, nvec):
    torch = torch_cuda()
    m = _model(dims, kinds, seed=sum(dims) + nvec)
    h = ham(m)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    x = torch.from_numpy(W.vector(h.D, 40 + nvec, nvec=nvec)).to("cuda", tdt)
    for transpose in (False, True):
        yv = h.apply_ex(x, kernel="general", transpose=transpose)
        ys = h.apply_ex(x, kernel="general", transpose=transpose, scalar=True)
        torch.cuda.synchronize()
        assert torch.equal(yv, ys), (dtype, nvec, transpose)
    yd = h.apply(x)
    assert torch.equal(yd, h.apply_ex(x, kernel="general"))
    xn = x.double().cpu().numpy()
    ref = oracle.apply(m.sites, m.terms, xn, nvec=nvec)
    check_close(yd.double().cpu().numpy(), ref, abs_bound(m, xn), TOL_F32 if dtype == "f32" else TOL_F64,
                f"{dims} {dtype} nvec={nvec}")


@pytest.mark.parametrize("dtype,nvec,offset", [("f32", 4, 1), ("f32", 4, 2), ("f32", 2, 1), ("f64", 2, 1)])
def test_misaligned_vectors_take_the_narrower_policy(dtype, nvec, offset):
    """x and y starting `offset` elements into their allocations (not aligned
    to the wide loads): the call runs the narrower policy, same results."""
    torch = torch_cuda()
    m = _model((2, 3, 2, 3, 2, 3, 2), None, seed=5)
    h = ham(m)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    n = h.D * nvec
    xb = torch.from_numpy(W.vector(n + offset, 9, nvec=1, normalize=False)).to("cuda", tdt)
    x = xb[offset:offset + n]
    yb = torch.full((n + offset,), float("nan"), dtype=tdt, device="cuda")
    y = yb[offset:offset + n]
    h.apply(x, out=y)
    ref = h.apply_ex(x.clone(), kernel="general", scalar=True)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    assert torch.isnan(yb[:offset]).all()


def test_complex_vectors_use_two_lanes_per_state():
    """A complex128 vector of a real H is the real apply on its (re, im)
    columns: the two-wide double-float policy, checked against the oracle."""
    torch = torch_cuda()
    m = _model((2, 3, 2, 3, 2, 3, 2, 3), None, seed=17)
    h = ham(m)
    xc = W.vector(h.D, 3) + 1j * W.vector(h.D, 4)
    y = h.apply(torch.from_numpy(xc).cuda()).cpu().numpy()
    ref = oracle.apply(m.sites, m.terms, xc)
    scale = abs_bound(m, np.abs(xc))
    err = np.abs(y - ref)
    assert (err <= TOL_F64 * scale + 1e-300).all()


@pytest.mark.parametrize("dtype,nvec", [("f32", 16), ("f32", 8), ("f64", 2), ("f64", 4)])
def test_batch_with_vector_lanes_equals_single_applies(dtype, nvec):
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch
    models = [W.xxz_spin1_chain(12, seed=71)] + W.disorder_ensemble(count=9, nmin=3, nmax=8, base_seed=72)
    hams = [ham(mm) for mm in models]
    tdt = torch.float32 if dtype == "f32" else torch.float64
    xs = [torch.from_numpy(W.vector(hh.D, 300 + i, nvec=nvec)).to("cuda", tdt) for i, hh in enumerate(hams)]
    ys = Batch(hams).apply(xs)
    torch.cuda.synchronize()
    for i, hh in enumerate(hams):
        assert torch.equal(hh.apply_ex(xs[i], kernel="general", scalar=True), ys[i]), i
    for i in (1, 2):
        xn = xs[i].double().cpu().numpy()
        ref = oracle.apply(models[i].sites, models[i].terms, xn, nvec=nvec)
        check_close(ys[i].double().cpu().numpy(), ref, abs_bound(models[i], xn),
                    TOL_F32 if dtype == "f32" else TOL_F64, models[i].name)
