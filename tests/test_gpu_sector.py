"""Sector plans (hm_create_sector, Sec. VI case 2, App. D) on the GPU against
the sector oracle, element by element: the projection P H P^T x for small
systems, the row-wise case-2 restatement on sampled rows of large ones, the
App. D worked update, several right-hand sides, FP32 storage, Lanczos inside a
sector, coefficient updates and the error codes."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, check_close, torch_cuda

pytestmark = pytest.mark.gpu


def _ham(sites, terms, total):
    from paper_2606_02169_gb300 import Hamiltonian
    return Hamiltonian(sites, terms, sector_total=total)


def _abs_scale(sites, terms, total, x, nvec=1):
    b = oracle.sector_basis(sites, total)
    Habs = abs(oracle.dense(sites, terms, sparse=True)).tocsr()[b][:, b]
    return np.asarray(Habs @ np.abs(np.asarray(x).reshape(b.size, nvec))).reshape(-1)


def _conserving(dims, kinds, seed):
    rng = np.random.default_rng(seed)
    n = len(dims)
    terms = []
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < 0.6 and kinds[i] == "spin" and kinds[j] == "spin":
                J, Jz = rng.uniform(-1, 1, 2)
                terms += [(i, "Sp", j, "Sm", J / 2), (i, "Sm", j, "Sp", J / 2), (i, "Sz", j, "Sz", Jz)]
            elif kinds[i] != kinds[j]:
                s, b = (i, j) if kinds[i] == "spin" else (j, i)
                g = rng.uniform(0.1, 1.0)
                terms += [(s, "Sm", b, "adag", g), (s, "Sp", b, "a", g)]
    for i in range(n):
        if kinds[i] == "spin":
            terms.append((i, "Sz", -1, "I", rng.uniform(-1, 1)))
            if dims[i] > 2:
                terms.append((i, "Sz2", -1, "I", rng.uniform(-1, 1)))
        else:
            terms.append((i, "N", -1, "I", rng.uniform(0.5, 1.5)))
    terms.append((0, "I", -1, "I", 0.25))     # a constant
    return [(k, d) for k, d in zip(kinds, dims)], terms


CASES = [((2, 3, 2, 4, 2), ("spin",) * 5),
         ((3, 2, 5, 2), ("spin", "spin", "boson", "spin")),
         ((6, 2, 2, 2, 2), ("boson", "spin", "spin", "spin", "spin")),
         ((2,) * 10, ("spin",) * 10)]


@pytest.mark.parametrize("dims,kinds", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sector_apply_matches_projection(dims, kinds, dtype):
    torch = torch_cuda()
    sites, terms = _conserving(dims, kinds, 7)
    for K in sorted({0, 1, sum(d - 1 for d in dims) // 2, sum(d - 1 for d in dims)}):
        h = _ham(sites, terms, K)
        n = oracle.sector_dimension(sites, K)
        assert h.D == n
        x = W.vector(n, 30 + K)
        if dtype == np.float32:
            x = x.astype(np.float32).astype(np.float64)
        ref = oracle.sector_apply(sites, terms, K, x)
        y = h.apply(torch.from_numpy(x).to("cuda", torch.float64 if dtype == np.float64 else torch.float32))
        torch.cuda.synchronize()
        check_close(y.double().cpu().numpy(), ref, _abs_scale(sites, terms, K, x),
                    TOL_F64 if dtype == np.float64 else TOL_F32, f"sector {dims} K={K}")


@pytest.mark.parametrize("nvec", [3, 11])
def test_sector_multiple_right_hand_sides(nvec):
    torch = torch_cuda()
    sites, terms = _conserving((2, 3, 2, 3, 2, 2), ("spin",) * 6, 8)
    K = 4
    h = _ham(sites, terms, K)
    x = W.vector(h.D, 5, nvec=nvec)
    ref = oracle.sector_apply(sites, terms, K, x, nvec=nvec)
    y = h.apply(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    check_close(y.cpu().numpy(), ref, _abs_scale(sites, terms, K, x, nvec), TOL_F64, "sector nvec")


def test_appendix_d_worked_update_on_gpu():
    """App. D: 4 spin-1/2 sites, zero magnetization, (J/2) S^+ S^- moving the
    source with packed index 3 into the target with packed index 5 (site
    labels in the main-text order, see tests/golden/appendix_d_sector.txt)."""
    torch = torch_cuda()
    J = 1.3
    h = _ham([("spin", 2)] * 4, [(1, "Sp", 3, "Sm", J / 2)], 2)
    assert h.D == 6
    x = torch.zeros(6, dtype=torch.float64, device="cuda")
    x[3] = 1.0
    y = h.apply(x).cpu().numpy()
    # the hop lands on packed index 5 alone; its value carries the
    # double-float coefficient (hi + lo float pair, ~2^-48 relative)
    assert np.array_equal(np.flatnonzero(y), [5])
    assert abs(y[5] - J / 2) <= 2.0 ** -45 * (J / 2)


def _chain(n, d, jz=1.0, h=0.3, seed=0):
    rng = np.random.default_rng(seed)
    sites = [("spin", d)] * n
    terms = []
    for i in range(n - 1):
        terms += [(i, "Sp", i + 1, "Sm", 0.5), (i, "Sm", i + 1, "Sp", 0.5), (i, "Sz", i + 1, "Sz", jz)]
    terms += [(0, "Sp", n - 1, "Sm", 0.5), (0, "Sm", n - 1, "Sp", 0.5), (0, "Sz", n - 1, "Sz", jz)]  # periodic
    for i in range(n):
        terms.append((i, "Sz", -1, "I", float(rng.uniform(-h, h))))
    return sites, terms


@pytest.mark.parametrize("n,d,dtype,tol", [(24, 2, np.float64, TOL_F64), (16, 3, np.float32, TOL_F32)])
def test_large_sector_sampled_rows(n, d, dtype, tol):
    """Periodic chains (the long bond exercises rank updates across all
    sites): sampled rows against the row-wise case-2 oracle."""
    torch = torch_cuda()
    sites, terms = _chain(n, d, seed=n)
    K = n * (d - 1) // 2
    h = _ham(sites, terms, K)
    assert h.D == oracle.sector_dimension(sites, K)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    x = W.torch_vector(h.D, 40, dtype=tdt)
    y = h.apply(x)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([rng.integers(0, h.D, size=300), [0, 1, h.D - 2, h.D - 1]]))
    xh = x.double().cpu().numpy()
    ref = oracle.sector_rows(sites, terms, K, xh, rows)
    got = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    bound = sum(abs(t[4]) * ((d - 1) / 2 + 1) ** 2 for t in terms) * np.abs(xh).max()
    check_close(got, ref, np.full(rows.size, bound), tol, f"sector chain n={n} d={d}")


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-10), (np.float32, 1e-5)])
def test_lanczos_in_the_zero_magnetization_sector(dtype, tol):
    torch = torch_cuda()
    m = W.heisenberg_ring(12)
    K = 6
    h = _ham(m.sites, m.terms, K)
    assert h.D == math.comb(12, 6)
    b = oracle.sector_basis(m.sites, K)
    H = oracle.dense(m.sites, m.terms, sparse=True).tocsr()[b][:, b].toarray().real
    e0 = np.linalg.eigvalsh(H)[0]
    v0 = torch.from_numpy(W.vector(h.D, 2)).to("cuda", torch.float64 if dtype == np.float64 else torch.float32)
    r = h.lanczos(v0, 120, reorth=True)
    assert abs(r["e0"] - e0) <= tol * abs(e0)


def test_sector_set_coefficients_matches_fresh_plan():
    torch = torch_cuda()
    sites, terms = _conserving((2, 3, 2, 3, 2), ("spin",) * 5, 11)
    K = 3
    h = _ham(sites, terms, K)
    c2 = [t[4] * (1.5 if k % 2 else -0.5) for k, t in enumerate(terms)]
    h.set_coefficients(c2)
    h2 = _ham(sites, [(t[0], t[1], t[2], t[3], c) for t, c in zip(terms, c2)], K)
    x = torch.from_numpy(W.vector(h.D, 3)).cuda()
    assert torch.equal(h.apply(x), h2.apply(x))


def test_sector_errors():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError, _capi as C
    sites = [("spin", 2)] * 4
    with pytest.raises(HmError) as e:
        _ham(sites, [(0, "Sx", -1, "I", 1.0)], 2)          # a lone Sx moves the digit sum
    assert e.value.code == C.HM_ERR_UNSUPPORTED
    with pytest.raises(HmError) as e:
        _ham(sites, [(0, "Sz", -1, "I", 1.0)], 5)          # empty sector
    assert e.value.code == C.HM_ERR_INVALID_ARG
    h = _ham(sites, [(0, "Sp", 1, "Sm", 1.0), (0, "Sm", 1, "Sp", 1.0)], 2)
    x = torch.zeros(h.D, dtype=torch.float64, device="cuda")
    for call in (lambda: h.apply_ex(x, kernel="tile"), lambda: h.apply_ex(x, mb=True), lambda: h.adjoint(x, x),
                 lambda: h.tune(1, torch.float64),
                 lambda: _ham(sites, [(0, "Sp", 1, "Sm", 1.0)], 2).adjoint(x, want_gcoef=False)):
        with pytest.raises(HmError) as e:
            call()
        assert e.value.code == C.HM_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        h.apply(torch.zeros(16, dtype=torch.float64, device="cuda")[:7])   # wrong length


def test_sector_adjoint_of_a_symmetric_term_list():
    """gx = H^T gy = H gy inside the sector (no coupling gradients)."""
    torch = torch_cuda()
    sites, terms = _chain(10, 2, seed=3)
    h = _ham(sites, terms, 5)
    gy = torch.from_numpy(W.vector(h.D, 8, nvec=2)).cuda()
    gx, g = h.adjoint(gy, want_gcoef=False)
    assert g is None and torch.equal(gx, h.apply(gy))
