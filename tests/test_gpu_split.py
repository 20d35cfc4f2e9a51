"""Top-site split (hm_apply_ex bit 14): the terms with an off-diagonal
operator on one of the leading T sites run as a second pass that adds to y,
visiting the low blocks with those digits varying fastest. Each pass rounds
once, so the result matches the oracle within the usual tolerances (not bit
for bit the one-pass kernel)."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, row_scale_bound, torch_cuda

pytestmark = pytest.mark.gpu

# every shape has at least three sites above its low block (a split's
# leading sites must be high sites)
SHAPES = [
    ((2, 3, 2, 3, 2, 3, 2, 3, 2, 3, 2, 3, 2), None),
    ((3, 2, 4, 2, 3, 2, 5, 2, 2, 3, 2, 2), None),
    ((5, 3, 2, 3) + (2,) * 11, [W.BOSON] + [W.SPIN] * 14),   # boson on top
    ((2,) * 12 + (9,), [W.SPIN] * 12 + [W.BOSON]),
]


def _with_top_hops(m, T):
    """m plus one hop term on each of the leading T sites (coupled to the
    last site's Sz), so that both passes of a T-site split have terms."""
    kinds = [k for k, _ in m.sites]
    n = len(m.sites)
    extra = []
    for k in range(T):
        if kinds[k] == W.BOSON:
            extra += [(k, "a", n - 1, "Sz" if kinds[n - 1] == W.SPIN else "N", 0.37),
                      (k, "adag", n - 1, "Sz" if kinds[n - 1] == W.SPIN else "N", 0.37)]
        else:
            extra.append((k, "Sx", n - 1, "Sz" if kinds[n - 1] == W.SPIN else "N", 0.41 + 0.1 * k))
    return W.Model(m.name + "_tophops", m.sites, m.terms + extra)


@pytest.mark.parametrize("dims,kinds", SHAPES)
@pytest.mark.parametrize("T", [1, 2, 3])
@pytest.mark.parametrize("dtype,nvec", [("f64", 1), ("f32", 1), ("f64", 2), ("f32", 4)])
def test_split_matches_oracle(dims, kinds, T, dtype, nvec):
    torch = torch_cuda()
    m = _with_top_hops(W.random_model(list(dims), kinds, nterms=40, seed=7 * T + len(dims)), T)
    h = ham(m)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    x = torch.from_numpy(W.vector(h.D, 11 + T, nvec=nvec)).to("cuda", tdt)
    xn = x.double().cpu().numpy()
    tol = TOL_F32 if dtype == "f32" else TOL_F64
    for transpose in (False, True):
        y = h.apply_ex(x, kernel="general", split=True, split_sites=T, transpose=transpose)
        y2 = h.apply_ex(x, kernel="general", split=True, split_sites=T, transpose=transpose)
        torch.cuda.synchronize()
        assert torch.equal(y, y2), "not reproducible"
        if transpose:
            Hd = oracle.dense(m.sites, m.terms, sparse=True).T.tocsr()
            ref = np.asarray(Hd @ xn.reshape(h.D, nvec)).reshape(-1)
        else:
            ref = oracle.apply(m.sites, m.terms, xn, nvec=nvec)
        check_close(y.double().cpu().numpy(), ref, abs_bound(m, xn) if not transpose else
                    np.asarray(abs(Hd) @ np.abs(xn).reshape(h.D, nvec)).reshape(-1), tol,
                    f"{dims} T={T} {dtype} nvec={nvec} transpose={transpose}")


def test_split_options_combine():
    """The split with the prefetching and register-capped first pass, each
    elements-per-thread value, and one right-hand side per lane."""
    torch = torch_cuda()
    m = W.random_model([2, 3, 2, 3, 2, 3, 2, 3, 2, 3, 2, 3, 2], None, nterms=40, seed=3)
    h = ham(m)
    x = torch.from_numpy(W.vector(h.D, 5, nvec=2)).cuda()
    xn = x.cpu().numpy()
    ref = oracle.apply(m.sites, m.terms, xn, nvec=2)
    scale = abs_bound(m, xn)
    for kw in (dict(prefetch=True, s=4), dict(prefetch=True, s=8, mb=True), dict(s=2), dict(s=6, mb=True),
               dict(scalar=True), dict(s=3, scalar=True)):
        y = h.apply_ex(x, kernel="general", split=True, split_sites=2, **kw)
        check_close(y.cpu().numpy(), ref, scale, TOL_F64, str(kw))


def test_split_rejected_without_a_second_pass():
    torch = torch_cuda()
    from paper_2606_02169_gb300._capi import HmError
    # only diagonal terms: nothing moves a leading digit
    sites = [(W.SPIN, 2)] * 8
    terms = [(i, "Sz", i + 1, "Sz", 1.0) for i in range(7)]
    from paper_2606_02169_gb300 import Hamiltonian
    h = Hamiltonian(sites, terms)
    x = torch.ones(h.D, dtype=torch.float64, device="cuda")
    with pytest.raises(HmError):
        h.apply_ex(x, kernel="general", split=True, split_sites=1)
    # every term moves the leading digit: pass A would be empty
    h2 = Hamiltonian(sites, [(0, "Sp", 1, "Sm", 0.5), (0, "Sm", 1, "Sp", 0.5)])
    with pytest.raises(HmError):
        h2.apply_ex(x, kernel="general", split=True, split_sites=1)
    # a split must not be combined with another kernel or native FP64
    h3 = ham(W.random_model([2, 3, 2, 3, 2, 3], None, nterms=20, seed=1))
    x3 = torch.ones(h3.D, dtype=torch.float64, device="cuda")
    with pytest.raises(HmError):
        h3.apply_ex(x3, kernel="general", split=True, native_f64=True)


def test_split_on_tavis_cummings_sampled_rows():
    """The split sized from the vector (Tavis-Cummings N = 20, D = 2^26,
    FP64: the four leading spins' hops reach 32 MiB or more) on sampled rows,
    and within rounding of the one-pass kernel."""
    torch = torch_cuda()
    m = W.tavis_cummings(20, 64, seed=7)
    h = ham(m)
    seed = 13
    x = W.torch_hashed_vector(h.D, seed, dtype=torch.float64)
    y = h.apply_ex(x, kernel="general", split=True)
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([[0, 1, h.D - 1, h.D // 2], rng.integers(0, h.D, size=3000)]))
    ref = oracle.rows_hashed(m.sites, m.terms, seed, rows, nthreads=oracle.max_threads())
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    check_close(got, ref, np.full(rows.size, row_scale_bound(m, 0.5)), TOL_F64, "TC N=20 split")
    yf = h.apply_ex(x, kernel="general")
    torch.cuda.synchronize()
    err = (y - yf).abs().max().item() / yf.abs().max().item()
    assert err < 1e-13
