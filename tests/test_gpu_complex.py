"""Complex storage (HM_C128 / HM_C64) of a real H and the time evolution
y = exp(-i t H) x (hm_evolve, Sec. VII exact propagation), on the GPU through
the C ABI, against the oracle: complex applies (full basis, sector, several
right-hand sides, batch), complex coupling gradients, Lanczos from a complex
start vector, hm_evolve against the dense-exponential oracle (full basis and
sector, FP64 and FP32, stored and rebuilt Krylov bases), a product-state
evolution at D = 2^22 checked on sampled entries against per-site closed
forms, unitarity and time reversal at scale, and the error codes."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_matrix, torch_cuda

pytestmark = pytest.mark.gpu


def _ham(sites, terms, total=None):
    from paper_2606_02169_gb300 import Hamiltonian
    return Hamiltonian(sites, terms, sector_total=total)


def _cx(D, seed, nvec=1):
    return W.vector(D, seed, nvec=nvec) + 1j * W.vector(D, seed + 101, nvec=nvec)


def _close(got, ref, scale, tol, what):
    err = np.abs(np.asarray(got) - np.asarray(ref))
    bad = np.flatnonzero(err > tol * scale + 1e-300)
    assert bad.size == 0, f"{what}: {bad.size} out of tolerance, worst {err[bad[:3]]} vs {scale[bad[:3]]}"


MODELS = [W.random_model([3, 2, 4, 2, 3], None, nterms=24, seed=11),
          W.random_model([2, 5, 2, 3], ["spin", "boson", "spin", "spin"], nterms=20, seed=12)]


@pytest.mark.parametrize("m", MODELS, ids=["spins", "spin_boson"])
@pytest.mark.parametrize("cdt,tol", [("complex128", TOL_F64), ("complex64", TOL_F32)])
@pytest.mark.parametrize("nvec", [1, 3])
def test_complex_apply_matches_oracle(m, cdt, tol, nvec):
    torch = torch_cuda()
    h = _ham(m.sites, m.terms)
    x = _cx(h.D, 5, nvec)
    xt = torch.from_numpy(x).to("cuda", getattr(torch, cdt))
    y = h.apply(xt).cpu().numpy()
    xr = xt.cpu().numpy().astype(np.complex128)
    ref = oracle.apply(m.sites, m.terms, xr, nvec=nvec)
    H = abs_matrix(m)
    scale = np.asarray(H @ np.abs(xr).reshape(h.D, nvec)).reshape(-1)
    _close(y, ref, scale, tol, f"{cdt} nvec={nvec}")


def test_complex_apply_is_the_real_apply_of_the_pairs():
    torch = torch_cuda()
    m = MODELS[0]
    h = _ham(m.sites, m.terms)
    x = torch.from_numpy(_cx(h.D, 7, 2)).cuda()
    y = torch.view_as_real(h.apply(x)).reshape(-1)
    yr = h.apply(torch.view_as_real(x).reshape(-1).contiguous())
    assert torch.equal(y, yr)


def test_complex_sector_apply_matches_oracle():
    torch = torch_cuda()
    sites = [("spin", 2), ("spin", 3), ("spin", 2), ("spin", 2), ("spin", 3)]
    terms = []
    for i in range(5):
        j = (i + 1) % 5
        a, b = min(i, j), max(i, j)
        terms += [(a, "Sp", b, "Sm", 0.4 + 0.1 * i), (a, "Sm", b, "Sp", 0.4 + 0.1 * i), (a, "Sz", b, "Sz", 0.7)]
        terms.append((i, "Sz", -1, "I", 0.2 * i - 0.3))
    h = _ham(sites, terms, 3)
    x = _cx(h.D, 9, 2)
    y = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.sector_apply(sites, terms, 3, x, nvec=2)
    assert np.allclose(y, ref, rtol=0, atol=TOL_F64 * np.abs(ref).max() * 10)


def test_complex_batch_equals_single_applies():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch
    hams = [_ham(mm.sites, mm.terms) for mm in W.disorder_ensemble(count=5, nmin=3, nmax=6, base_seed=81)]
    xs = [torch.from_numpy(_cx(h.D, 20 + i, 2)).cuda() for i, h in enumerate(hams)]
    ys = Batch(hams).apply(xs)
    for h, x, y in zip(hams, xs, ys):
        assert torch.equal(h.apply(x), y)


def test_complex_coupling_gradients_are_the_real_part():
    """gcoef[t] = Re sum_v <gy_v| O_t |x_v>, O_t x from one-term oracle applies."""
    torch = torch_cuda()
    m = MODELS[0]
    h = _ham(m.sites, m.terms)
    gy, x = _cx(h.D, 31), _cx(h.D, 33)
    _, g = h.adjoint(torch.from_numpy(gy).cuda(), torch.from_numpy(x).cuda(), want_gx=False)
    g = g.cpu().numpy()
    for t, (i, oi, j, oj, _) in enumerate(m.terms):
        ox = oracle.apply(m.sites, [(i, oi, j, oj, 1.0)], x)
        want = np.real(np.vdot(gy, ox))
        assert abs(g[t] - want) <= 1e-11 * (np.abs(gy).sum() * np.abs(x).max() * 8 + 1)


def test_lanczos_from_a_complex_start_vector():
    torch = torch_cuda()
    mm = W.heisenberg_ring(10)
    h = _ham(mm.sites, mm.terms)
    e_exact = np.linalg.eigvalsh(oracle.dense(mm.sites, mm.terms).real)[0]
    v0 = torch.from_numpy(_cx(h.D, 41)).cuda()
    r = h.lanczos(v0, 80, reorth=True, ritz_vector=True)
    assert abs(r["e0"] - e_exact) < 1e-9 * abs(e_exact)
    psi = r["psi0"]
    res = h.apply(psi) - r["e0"] * psi
    assert float(torch.linalg.vector_norm(res)) < 1e-6


HERMITIAN = [W.random_model([3, 2, 4, 2, 3], None, nterms=16, seed=13, hermitian=True),
             W.random_model([2, 5, 2, 3], ["spin", "boson", "spin", "spin"], nterms=16, seed=14, hermitian=True)]
EVOLVE_CASES = [(HERMITIAN[0], 0.8), (HERMITIAN[1], 1.5)]


@pytest.mark.parametrize("case", [0, 1])
@pytest.mark.parametrize("cdt,tol", [("complex128", 1e-10), ("complex64", 2e-5)])
@pytest.mark.parametrize("recompute", [False, True])
def test_evolve_matches_the_dense_exponential(case, cdt, tol, recompute):
    torch = torch_cuda()
    m, t = EVOLVE_CASES[case]
    h = _ham(m.sites, m.terms)
    x = torch.from_numpy(_cx(h.D, 51)).to("cuda", getattr(torch, cdt))
    y, err = h.evolve(x, t, m=30, substeps=4, recompute=recompute)
    ref = oracle.evolve(m.sites, m.terms, x.cpu().numpy().astype(np.complex128), t)
    nrm = np.linalg.norm(ref)
    assert np.linalg.norm(y.cpu().numpy() - ref) <= tol * nrm
    assert err < 1e-8 * nrm


def test_stored_and_rebuilt_bases_agree_bit_for_bit():
    torch = torch_cuda()
    m = HERMITIAN[0]
    h = _ham(m.sites, m.terms)
    x = torch.from_numpy(_cx(h.D, 61)).cuda()
    a, _ = h.evolve(x, 0.6, m=20, substeps=3, reorth=True)
    b, _ = h.evolve(x, 0.6, m=20, substeps=3, reorth=True, recompute=True)
    assert torch.equal(a, b)


def test_sector_evolution_matches_the_oracle():
    torch = torch_cuda()
    sites = [("spin", 2)] * 8
    terms = []
    for i in range(8):
        j = (i + 1) % 8
        a, b = min(i, j), max(i, j)
        terms += [(a, "Sp", b, "Sm", 0.5), (a, "Sm", b, "Sp", 0.5), (a, "Sz", b, "Sz", 1.1)]
        terms.append((i, "Sz", -1, "I", 0.15 * ((3 * i) % 5)))
    h = _ham(sites, terms, 4)
    x = _cx(h.D, 71)
    y, _ = h.evolve(torch.from_numpy(x).cuda(), 2.0, m=40, substeps=2)
    ref = oracle.evolve(sites, terms, x, 2.0, sector_total=4)
    assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_product_state_evolution_at_scale():
    """22 spins-1/2 in transverse fields h_k S_x plus longitudinal g_k S_z
    (no couplings): exp(-i t H) of a product state is the product of the
    single-site evolutions (oracle.evolve on one site each); sampled entries
    of the D = 2^22 result are compared with those products, and the whole
    vector keeps its norm."""
    torch = torch_cuda()
    n = 22
    rng = np.random.default_rng(5)
    hs, gs = rng.uniform(0.3, 1.2, n), rng.uniform(-0.5, 0.5, n)
    sites = [("spin", 2)] * n
    terms = [(k, "Sx", -1, "I", float(hs[k])) for k in range(n)] + [(k, "Sz", -1, "I", float(gs[k]))
                                                                    for k in range(n)]
    h = _ham(sites, terms)
    loc = [np.array([np.cos(0.3 * k), np.sin(0.3 * k) * np.exp(0.5j * k)]) for k in range(n)]
    t = 1.7
    out = [oracle.evolve([("spin", 2)], [(0, "Sx", -1, "I", float(hs[k])), (0, "Sz", -1, "I", float(gs[k]))],
                         loc[k], t) for k in range(n)]
    # the product state on the device (site 0 most significant)
    x = torch.ones(1, dtype=torch.complex128, device="cuda")
    for k in range(n):
        x = torch.kron(x, torch.from_numpy(loc[k]).cuda())
    y, err = h.evolve(x, t, m=40, substeps=6)
    idx = np.unique(np.concatenate([rng.integers(0, h.D, 400), [0, h.D - 1]]))
    got = y[torch.from_numpy(idx).cuda()].cpu().numpy()
    for F, g in zip(idx, got):
        want = 1.0 + 0j
        for k in range(n):
            want *= out[k][(F >> (n - 1 - k)) & 1]
        assert abs(g - want) < 1e-9, (F, g, want)
    assert abs(float(torch.linalg.vector_norm(y)) - 1.0) < 1e-10


def test_time_reversal_at_scale():
    torch = torch_cuda()
    mm = W.ferrimagnet_chain(16)
    h = _ham(mm.sites, mm.terms)
    x = torch.from_numpy(_cx(h.D, 91)).cuda()
    x = x / torch.linalg.vector_norm(x)
    y, e1 = h.evolve(x, 0.5, m=30, substeps=2)
    z, e2 = h.evolve(y, -0.5, m=30, substeps=2)
    assert abs(float(torch.linalg.vector_norm(y)) - 1.0) < 1e-10
    assert float(torch.linalg.vector_norm(z - x)) < 1e-9
    assert e1 < 1e-9 and e2 < 1e-9


def test_evolve_errors():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError, _capi as C
    m = HERMITIAN[0]
    h = _ham(m.sites, m.terms)
    x = torch.from_numpy(_cx(h.D, 3)).cuda()
    for kw in ({"m": 0}, {"m": 129}, {"substeps": 0}):
        with pytest.raises(HmError) as e:
            h.evolve(x, 0.1, **kw)
        assert e.value.code == C.HM_ERR_INVALID_ARG
    with pytest.raises(HmError) as e:
        h.evolve(x, 0.1, out=x)
    assert e.value.code == C.HM_ERR_ALIAS
    nh = _ham([("spin", 2), ("spin", 2)], [(0, "Sp", 1, "Sm", 1.0)])     # not self-adjoint
    with pytest.raises(HmError) as e:
        nh.evolve(torch.zeros(4, dtype=torch.complex128, device="cuda"), 0.1)
    assert e.value.code == C.HM_ERR_NOT_HERMITIAN
    with pytest.raises(ValueError):
        h.evolve(x.real.contiguous(), 0.1)
    z = torch.zeros_like(x)
    y, err = h.evolve(z, 0.3)
    assert float(torch.linalg.vector_norm(y)) == 0.0 and err == 0.0


# ---------------------------------------------------------------------------
# complex H (imaginary matrix elements from Sy factors)
# ---------------------------------------------------------------------------

def _dm_chain(n=7, d=2, J=1.0, Dm=0.45, hy=0.3, seed=0):
    """Heisenberg chain with a Dzyaloshinskii-Moriya term D (Sx_i Sy_j - Sy_i
    Sx_j) and a transverse Sy field: Hermitian, with imaginary elements."""
    rng = np.random.default_rng(seed)
    sites = [("spin", d)] * n
    terms = []
    for i in range(n - 1):
        j = i + 1
        terms += [(i, "Sx", j, "Sx", J), (i, "Sy", j, "Sy", J), (i, "Sz", j, "Sz", J * 0.8),
                  (i, "Sx", j, "Sy", Dm), (i, "Sy", j, "Sx", -Dm)]
    for i in range(n):
        terms += [(i, "Sy", -1, "I", hy * rng.uniform(0.5, 1.5)), (i, "Sz", -1, "I", 0.2 * rng.normal())]
    return sites, terms


CX_MODELS = [_dm_chain(7, 2, seed=1), _dm_chain(5, 3, seed=2),
             ([("spin", 2), ("boson", 4), ("spin", 3)],
              [(0, "Sy", 1, "N", 0.7), (2, "Sy", -1, "I", 0.4), (0, "Sm", 1, "adag", 0.5), (0, "Sp", 1, "a", 0.5),
               (2, "Sx", 0, "Sy", 0.3), (1, "N", -1, "I", 1.1)])]


@pytest.mark.parametrize("case", [0, 1, 2])
@pytest.mark.parametrize("cdt,tol", [("complex128", TOL_F64), ("complex64", TOL_F32)])
@pytest.mark.parametrize("nvec", [1, 2])
def test_complex_h_apply_matches_oracle(case, cdt, tol, nvec):
    torch = torch_cuda()
    sites, terms = CX_MODELS[case]
    h = _ham(sites, terms)
    x = _cx(h.D, 13, nvec)
    xt = torch.from_numpy(x).to("cuda", getattr(torch, cdt))
    y = h.apply(xt).cpu().numpy()
    xr = xt.cpu().numpy().astype(np.complex128)
    ref = oracle.apply(sites, terms, xr, nvec=nvec)
    H = abs(oracle.dense(sites, terms, sparse=True))
    scale = np.asarray(H @ np.abs(xr).reshape(h.D, nvec)).reshape(-1)
    assert np.abs(ref.imag).max() > 0
    _close(y, ref, scale, tol, f"complex H case {case} {cdt}")


def test_complex_h_adjoint_is_the_conjugate_transpose():
    torch = torch_cuda()
    sites = [("spin", 2), ("spin", 3), ("spin", 2)]
    terms = [(0, "Sy", 1, "Sp", 0.7), (1, "Sy", -1, "I", -0.4), (0, "Sx", 2, "Sy", 0.5), (2, "Sm", -1, "I", 0.3)]
    h = _ham(sites, terms)                   # not self-adjoint
    gy = _cx(h.D, 17)
    gx, _ = h.adjoint(torch.from_numpy(gy).cuda(), want_gcoef=False)
    Hd = oracle.dense(sites, terms).conj().T
    assert np.allclose(gx.cpu().numpy(), Hd @ gy, rtol=0, atol=1e-13)


def test_complex_h_lanczos_and_evolution():
    torch = torch_cuda()
    sites, terms = CX_MODELS[0]
    h = _ham(sites, terms)
    H = oracle.dense(sites, terms)
    assert np.abs(H - H.conj().T).max() < 1e-14 and np.abs(H.imag).max() > 0
    e_exact = np.linalg.eigvalsh(H)[0]
    r = h.lanczos(torch.from_numpy(_cx(h.D, 19)).cuda(), 100, reorth=True, ritz_vector=True)
    assert abs(r["e0"] - e_exact) < 1e-9 * abs(e_exact)
    psi = r["psi0"]
    assert float(torch.linalg.vector_norm(h.apply(psi) - r["e0"] * psi)) < 1e-6
    x = _cx(h.D, 23)
    for cdt, tol in (("complex128", 1e-10), ("complex64", 2e-5)):
        xt = torch.from_numpy(x).to("cuda", getattr(torch, cdt))
        y, err = h.evolve(xt, 1.3, m=30, substeps=3)
        ref = oracle.evolve(sites, terms, xt.cpu().numpy().astype(np.complex128), 1.3)
        assert np.linalg.norm(y.cpu().numpy() - ref) <= tol * np.linalg.norm(ref), cdt


def test_complex_h_coefficient_updates_and_tuning():
    torch = torch_cuda()
    sites, terms = CX_MODELS[1]
    h = _ham(sites, terms)
    x = torch.from_numpy(_cx(h.D, 29)).cuda()
    # switch every Sy-carrying coefficient off: the plan becomes real
    c0 = [t[4] for t in terms]
    c1 = [0.0 if "Sy" in (t[1], t[3]) and not (t[1] == "Sy" and t[3] == "Sy") else t[4] for t in terms]
    h.set_coefficients(c1)
    real_terms = [(t[0], t[1], t[2], t[3], c) for t, c in zip(terms, c1)]
    h.apply(torch.zeros(h.D, dtype=torch.float64, device="cuda"))          # real storage works again
    assert torch.equal(h.apply(x), _ham(sites, real_terms).apply(x))
    from paper_2606_02169_gb300 import HmError, _capi as C
    with pytest.raises(HmError) as e:           # the zeroed Sy terms have no real gradient
        h.adjoint(x, x)
    assert e.value.code == C.HM_ERR_UNSUPPORTED
    h.set_coefficients(c0)
    assert torch.equal(h.apply(x), _ham(sites, terms).apply(x))
    h.tune(1, torch.complex128)
    ref = oracle.apply(sites, terms, x.cpu().numpy())
    assert np.allclose(h.apply(x).cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_complex_h_errors():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch, HmError, _capi as C
    sites, terms = CX_MODELS[0]
    h = _ham(sites, terms)
    xr = torch.zeros(h.D, dtype=torch.float64, device="cuda")
    xc = torch.zeros(h.D, dtype=torch.complex128, device="cuda")
    with pytest.raises(HmError) as e:
        h.apply(xr)
    assert e.value.code == C.HM_ERR_COMPLEX_REQUIRED
    with pytest.raises(HmError) as e:
        h.apply_ex(xc, prefetch=True)          # complex H: bits 0, 1, 4 and 13 only
    assert e.value.code == C.HM_ERR_UNSUPPORTED
    with pytest.raises(HmError) as e:
        h.apply_ex(xr)
    assert e.value.code == C.HM_ERR_COMPLEX_REQUIRED
    with pytest.raises(HmError) as e:
        h.adjoint(xc, xc)
    assert e.value.code == C.HM_ERR_UNSUPPORTED
    with pytest.raises(HmError) as e:
        Batch([h])
    assert e.value.code == C.HM_ERR_INVALID_ARG
    with pytest.raises(HmError) as e:
        _ham(sites, terms, 3)
    assert e.value.code in (C.HM_ERR_UNSUPPORTED,)
