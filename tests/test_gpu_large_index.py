"""64-bit indexing at full size: sampled-row parity past 2^31 states in FP64
storage and past 2^32 states in FP32 storage, and a fixed-magnetization
sector of more than 2^31 retained states (64-bit rank deltas). The vectors
are synthesised on the device by the counter-based generator (splitmix64)
that the oracle implements on its own, so no vector is copied to the host;
each test first checks that the device vector holds the generator's values."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, check_close, ham, row_scale_bound, torch_cuda

pytestmark = pytest.mark.gpu


def _rows(dims, D, rng, n_random):
    mult, _ = oracle.multipliers(dims)
    rows = {r for r in (0, D - 1, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 1, 2 ** 32) if r < D}
    for _ in range(2000):   # digits at their bounds (every channel's admissibility edge)
        digits = [int(rng.choice([0, d - 1, rng.integers(0, d)])) for d in dims]
        rows.add(int(np.dot(digits, mult)))
    rows = np.unique(np.concatenate([np.array(sorted(rows), dtype=np.int64), rng.integers(0, D, size=n_random)]))
    return rows


def _mixed_chain(n_spin1, seed):
    """One spin-1/2 site ahead of an XXZ spin-1 chain of n_spin1 sites (bond
    0-1 Heisenberg): D = 2 * 3^n_spin1."""
    m = W.xxz_spin1_chain(n_spin1, seed=seed)
    terms = [(t[0] + 1, t[1], t[2] + 1 if t[2] >= 0 else -1, t[3], t[4]) for t in m.terms]
    return W.Model(f"half_plus_spin1_chain_{n_spin1}", [("spin", 2)] + m.sites, terms + W.heisenberg_bond(0, 1, 0.7))


def _check_device_vector(x, seed, f32):
    torch = torch_cuda()
    D = x.numel()
    probe = np.unique(np.array([0, 1, D // 3, D - 2, D - 1, min(D - 1, 2 ** 31 + 5), min(D - 1, 2 ** 32 + 9)]))
    got = x[torch.from_numpy(probe).cuda()].double().cpu().numpy()
    assert np.array_equal(got, oracle.hashed_values(seed, probe, f32))


def _sampled(model, dtype, seed, n_random, tol, kernels):
    torch = torch_cuda()
    h = ham(model)
    D = h.D
    f32 = dtype == np.float32
    tdt = torch.float32 if f32 else torch.float64
    x = W.torch_hashed_vector(D, seed, dtype=tdt)
    _check_device_vector(x, seed, f32)
    rng = np.random.default_rng(seed)
    rows = _rows(model.dims, D, rng, n_random)
    ref = oracle.rows_hashed(model.sites, model.terms, seed, rows, f32=f32, nthreads=oracle.max_threads())
    scale = np.full(rows.size, row_scale_bound(model, 0.5))
    ridx = torch.from_numpy(rows).cuda()
    for kernel in kernels:
        y = h.apply(x) if kernel is None else h.apply_ex(x, kernel=kernel)
        got = y[ridx].double().cpu().numpy()
        del y
        torch.cuda.empty_cache()
        check_close(got, ref, scale, tol, f"{model.name} {kernel}")
    from paper_2606_02169_gb300 import _capi
    assert _capi.device_status() == 0


def test_fp64_past_2_31_states():
    """D = 2 * 3^19 = 2.32e9 > 2^31, FP64 storage (x, y and the split copy:
    56 GB on the device)."""
    m = _mixed_chain(19, seed=77)
    assert oracle.dimension(m.sites) > 2 ** 31
    _sampled(m, np.float64, 31, 20000, TOL_F64, [None, "staged"])


def test_fp32_past_2_32_states():
    """D = 2 * 3^20 = 6.97e9 > 2^32, FP32 storage (x and y: 56 GB)."""
    m = _mixed_chain(20, seed=78)
    assert oracle.dimension(m.sites) > 2 ** 32
    _sampled(m, np.float32, 32, 20000, TOL_F32, [None])


def test_sector_past_2_31_retained_states():
    """Periodic spin-1/2 Heisenberg chain N = 34 in M = 0: C(34, 17) = 2.33e9
    retained states (64-bit rank deltas), FP32 storage, sampled packed rows
    against the sector oracle's case-2 restatement."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian
    n = 34
    sites = [("spin", 2)] * n
    terms = []
    for i in range(n):
        j = (i + 1) % n
        terms += [(i, "Sp", j, "Sm", 0.5), (i, "Sm", j, "Sp", 0.5), (i, "Sz", j, "Sz", 1.0)]
    h = Hamiltonian(sites, terms, sector_total=n // 2)
    assert h.D == 2333606220
    seed = 34
    x = W.torch_hashed_vector(h.D, seed, dtype=torch.float32)
    _check_device_vector(x, seed, True)
    y = h.apply(x)
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([[0, 1, h.D - 1, 2 ** 31 - 1, 2 ** 31], rng.integers(0, h.D, size=300)]))
    got = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    ref = oracle.sector_rows(sites, terms, n // 2, None, rows, seed=seed, f32=True)
    # each row sums at most 2 n hops and n diagonal bonds of |x| <= 1/2
    check_close(got, ref, np.full(rows.size, 2.0 * n * 0.5), TOL_F32, "sector N=34")
