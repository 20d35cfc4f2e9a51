"""GPU parity of y = H x (hm_apply through the C ABI) against the CPU oracle,
element by element, on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, apply_abs_bound, check_close, ham, row_abs_bound, torch_cuda

pytestmark = pytest.mark.gpu

# dims chosen to hit: no high sites; 1-2 high sites; ragged low blocks;
# a boson as a high site and as the low block; single sites of 4500 and of
# 9000 levels (the latter above the 8192-state low-block bound)
SMALL = [
    ((2,), None),
    ((3,), None),
    ((5, 7), None),
    ((2, 3, 4), None),
    ((3, 2, 5, 2, 3, 4, 2, 3, 2), None),                       # D=8640, B=2880 (ragged)
    ((2,) * 14, None),                                           # D=16384, 2 high sites
    ((64, 2, 2, 2, 2, 2, 2, 2), ["boson"] + ["spin"] * 7),       # boson high
    ((2, 2, 2, 2, 2, 2, 2, 64), ["spin"] * 7 + ["boson"]),       # boson in the low block
    ((3, 5, 2, 7, 3, 2, 2, 3), ["spin", "boson", "spin", "boson", "spin", "spin", "spin", "spin"]),
    ((4500,), ["boson"]),                                        # one large site
    ((9000,), ["boson"]),                                        # one site above the block bound
    ((4, 4500), ["spin", "boson"]),
]


def _scale(m, x):
    """(|H||x|)_F where the Kronecker assembly is cheap; for a site of several
    thousand levels (dense local matrices) the per-term bound from the
    row-wise oracle on |x|."""
    if max(m.dims) > 1024:
        return apply_abs_bound(m, x, nvec=x.size // oracle.dimension(m.sites))
    return abs_bound(m, x)


def _run(model, x_np, dtype, nvec=1, native=False):
    torch = torch_cuda()
    h = ham(model)
    x = torch.from_numpy(x_np).to("cuda", torch.float64 if dtype == np.float64 else torch.float32)
    y = h.apply_ex(x, native_f64=True) if native else h.apply(x)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("dims,kinds", SMALL)
@pytest.mark.parametrize("seed", [0, 1])
def test_random_models_fp64(dims, kinds, seed):
    m = W.random_model(list(dims), kinds, nterms=28, seed=seed)
    D = oracle.dimension(m.sites)
    x = W.vector(D, seed + 100)
    ref = oracle.apply(m.sites, m.terms, x)
    got = _run(m, x, np.float64)
    check_close(got, ref, _scale(m, x), TOL_F64, f"fp64 {dims}")


@pytest.mark.parametrize("dims,kinds", SMALL[3:8])
def test_random_models_native_fp64(dims, kinds):
    m = W.random_model(list(dims), kinds, nterms=28, seed=5)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 7)
    ref = oracle.apply(m.sites, m.terms, x)
    got = _run(m, x, np.float64, native=True)
    check_close(got, ref, abs_bound(m, x), 1e-13, f"native fp64 {dims}")


@pytest.mark.parametrize("dims,kinds", SMALL)
def test_random_models_fp32(dims, kinds):
    """Kernel error: oracle applied to the FP32-rounded x."""
    m = W.random_model(list(dims), kinds, nterms=28, seed=3)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 9).astype(np.float32).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x)
    got = _run(m, x, np.float32)
    check_close(got, ref, _scale(m, x), TOL_F32, f"fp32 {dims}")


@pytest.mark.parametrize("nvec", [2, 3, 4, 8, 16])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_multiple_right_hand_sides(nvec, dtype):
    m = W.random_model([3, 2, 4, 2, 3, 2, 5, 2], None, nterms=30, seed=11)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 12, nvec=nvec).astype(dtype).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x, nvec=nvec)
    got = _run(m, x, dtype, nvec=nvec)
    tol = TOL_F64 if dtype == np.float64 else TOL_F32
    check_close(got, ref, abs_bound(m, x), tol, f"nvec={nvec}")


def test_misaligned_vectors_fall_back_to_scalar_access():
    torch = torch_cuda()
    m = W.random_model([2, 3, 2, 4, 2], None, nterms=20, seed=2)
    D = oracle.dimension(m.sites)
    nvec = 4
    x = W.vector(D, 3, nvec=nvec)
    h = ham(m)
    buf = torch.zeros(D * nvec + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(D * nvec + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(x).cuda()
    y = h.apply(buf[1:], out=out[1:])
    ref = oracle.apply(m.sites, m.terms, x, nvec=nvec)
    check_close(y.cpu().numpy(), ref, abs_bound(m, x), TOL_F64, "misaligned")


def test_bit_reproducible():
    torch = torch_cuda()
    m = W.ferrimagnet_chain(12)
    h = ham(m)
    x = torch.from_numpy(W.vector(h.D, 3)).cuda()
    a = h.apply(x).clone()
    b = h.apply(x)
    assert torch.equal(a, b)


# ---------------------------------------------------------------------------
# the workload shapes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_heisenberg_ring_n12(dtype):
    m = W.heisenberg_ring(12)
    x = W.vector(4096, 1).astype(dtype).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x)
    got = _run(m, x, dtype)
    check_close(got, ref, abs_bound(m, x), TOL_F64 if dtype == np.float64 else TOL_F32, "ring12")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_square_lattice_4x5_full_vector(dtype):
    m = W.square_lattice_xxz(4, 5, seed=4)
    D = 1 << 20
    x = W.vector(D, 5).astype(dtype).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x)
    got = _run(m, x, dtype)
    check_close(got, ref, abs_bound(m, x), TOL_F64 if dtype == np.float64 else TOL_F32, "4x5")


def boundary_rows(dims, rng, count):
    """Rows whose digits sit at the edges of their ranges (0 and d-1 mixed in),
    where admissibility tests matter most; plus the first and last rows."""
    D = oracle.dimension([("spin", d) for d in dims])
    mult, _ = oracle.multipliers(dims)
    rows = {0, D - 1}
    for _ in range(count):
        digits = [int(rng.choice([0, d - 1, rng.integers(0, d)])) for d in dims]
        rows.add(int(np.dot(digits, mult)))
    return np.array(sorted(rows), dtype=np.int64)


def sampled_parity(model, dtype, seed, n_random, tol):
    """Full-size apply in the launch configuration the benchmark times (the
    autotuned one), checked on sampled rows; the library-default launch of
    the same kernel must give the same y bit for bit."""
    torch = torch_cuda()
    h = ham(model)
    D = h.D
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    cfg = h.tune(1, tdt)
    x = W.torch_vector(D, seed, dtype=tdt)
    y = h.apply(x)
    kernel = {1: "general", 2: "tile", 3: "staged"}[cfg["kernel"]]
    extra = {} if kernel != "general" else dict(split=bool(cfg["split"]), split_sites=cfg["split_sites"],
                                                vinv=bool(cfg["vinv"]))
    y0 = h.apply_ex(x, kernel=kernel, small=bool(cfg["small"]), **extra)
    # (the prefetching, register-capped, elements-per-thread and lanes-per-
    # state variants sum like the default launch of the same form)
    torch.cuda.synchronize()
    assert torch.equal(y, y0), f"tuned launch {cfg} differs from the default launch of its kernel"
    del y0
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([rng.integers(0, D, size=n_random),
                                     boundary_rows(model.dims, rng, 2000)]))
    got = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    del y
    xh = x.cpu().numpy().astype(np.float64)
    del x
    torch.cuda.empty_cache()
    ref = oracle.rows(model.sites, model.terms, xh, rows)
    scale = row_abs_bound(model, xh, rows)
    return check_close(got, ref, scale, tol, model.name)


@pytest.mark.parametrize("dtype,tol", [(np.float64, TOL_F64), (np.float32, TOL_F32)])
def test_ferrimagnet_chain_n20_sampled(dtype, tol):
    sampled_parity(W.ferrimagnet_chain(20), dtype, 3, 100000, tol)


@pytest.mark.parametrize("dtype,tol", [(np.float64, TOL_F64), (np.float32, TOL_F32)])
def test_tavis_cummings_1e9_sampled(dtype, tol):
    sampled_parity(W.tavis_cummings(24, 64, seed=7), dtype, 8, 20000, tol)


@pytest.mark.parametrize("dtype,tol", [(np.float64, TOL_F64), (np.float32, TOL_F32)])
@pytest.mark.parametrize("model", [W.paper_c1_chain(), W.paper_c2_chain()], ids=["c1_spin1_pbc", "c2_mixed_pbc"])
def test_paper_table1_models_sampled(model, dtype, tol):
    """The paper's Sec. V testbeds C1 (D = 3^15) and C2 (D = 24^6), periodic."""
    sampled_parity(model, dtype, 13, 20000, tol)


def test_index_past_2_31_sampled():
    """D = 2 * 3^19 > 2^31: 64-bit source offsets and digit decoding."""
    m = W.xxz_spin1_chain(19, seed=77)
    m = W.Model("mixed_past_2_31", [("spin", 2)] + m.sites, [(t[0] + 1, t[1], t[2] + 1 if t[2] >= 0 else -1, t[3], t[4]) for t in m.terms] + W.heisenberg_bond(0, 1, 0.7))
    assert oracle.dimension(m.sites) > 2 ** 31
    sampled_parity(m, np.float32, 21, 20000, TOL_F32)


def test_boson_first_tavis_cummings_sampled():
    sampled_parity(W.tavis_cummings(14, 32, seed=5, boson_first=True), np.float64, 4, 20000, TOL_F64)


# ---------------------------------------------------------------------------
# invariants at full size
# ---------------------------------------------------------------------------

def test_excitation_number_conserved_tc():
    """TC conserves N_exc = n_b + number of up spins: a vector in one sector
    maps into that sector with exact zeros elsewhere (App. C channels)."""
    torch = torch_cuda()
    m = W.tavis_cummings(10, 16, seed=3)
    h = ham(m)
    D = h.D
    dims = m.dims
    idx = np.arange(D)
    nexc = np.zeros(D, dtype=np.int64)
    mult, _ = oracle.multipliers(dims)
    for k, d in enumerate(dims):
        nexc += (idx // mult[k]) % d
    x = np.where(nexc == 7, W.vector(D, 2), 0.0)
    y = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(y[nexc != 7] == 0.0)
    assert np.linalg.norm(y[nexc == 7]) > 0


# ---------------------------------------------------------------------------
# error behaviour through the C ABI
# ---------------------------------------------------------------------------

def test_alias_and_dtype_errors():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError, _capi as C
    h = ham(W.heisenberg_ring(4))
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(HmError) as e:
        h.apply(x, out=x)
    assert e.value.code == C.HM_ERR_ALIAS
    with pytest.raises(TypeError):
        h.apply(x.to(torch.float16))


def test_complex_term_list_needs_complex_storage():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError, _capi as C, Hamiltonian
    h = Hamiltonian([("spin", 3)], [(0, "Sy", -1, "I", 1.0)])   # imaginary elements: a complex plan
    with pytest.raises(HmError) as e:
        h.apply(torch.zeros(3, dtype=torch.float64, device="cuda"))
    assert e.value.code == C.HM_ERR_COMPLEX_REQUIRED
    h.apply(torch.zeros(3, dtype=torch.complex128, device="cuda"))
    # SySy is real and takes real storage
    Hamiltonian([("spin", 3), ("spin", 2)], [(0, "Sy", 1, "Sy", 1.0)]).apply(
        torch.zeros(6, dtype=torch.float64, device="cuda"))


def test_set_coefficients_matches_fresh_plan():
    torch = torch_cuda()
    m = W.square_lattice_xxz(3, 3, seed=8)
    h = ham(m)
    D = h.D
    rng = np.random.default_rng(0)
    c2 = rng.normal(size=len(m.terms))
    h.set_coefficients(c2)
    x = W.vector(D, 4)
    got = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.apply(m.sites, m.terms, x, coefs=c2)
    m2 = W.Model("c2", m.sites, [(t[0], t[1], t[2], t[3], float(c)) for t, c in zip(m.terms, c2)])
    check_close(got, ref, abs_bound(m2, x), TOL_F64, "set_coefficients")
