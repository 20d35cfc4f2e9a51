"""Complex H = H_re + i H_im in one pass (hm_apply_ex without bit 13, or
where hm_tune chose it): both real operators' sums of an element formed by
one thread and combined in registers. Each sum takes the real kernel's operations on the (re, im)
columns and the combination is the separate passes' one rounding, so the
one-pass result is bit-identical to the two real applies with their combine
(hm_apply_ex bit 13); both match the oracle, for H and H^dagger, FP32 and
FP64 storage, native FP64, inputs outside the double-float window, several
right-hand sides, several low blocks with a ragged last chunk, and vectors
that allow only the two-pass form."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, torch_cuda

pytestmark = pytest.mark.gpu


def _ham(sites, terms):
    from paper_2606_02169_gb300 import Hamiltonian
    return Hamiltonian(sites, terms)


def _cx(D, seed, nvec=1):
    return W.vector(D, seed, nvec=nvec) + 1j * W.vector(D, seed + 101, nvec=nvec)


def _dm(n, d, seed, ring=False):
    """Heisenberg chain with a Dzyaloshinskii-Moriya term, a transverse Sy
    field and a random Sz field (Hermitian, with imaginary elements)."""
    rng = np.random.default_rng(seed)
    sites = [("spin", d)] * n
    terms = []
    for i in range(n if ring else n - 1):
        a, b = sorted((i, (i + 1) % n))
        terms += [(a, "Sx", b, "Sx", 1.0), (a, "Sy", b, "Sy", 1.0), (a, "Sz", b, "Sz", 0.8),
                  (a, "Sx", b, "Sy", 0.35), (a, "Sy", b, "Sx", -0.35)]
    for i in range(n):
        terms += [(i, "Sy", -1, "I", 0.3 * rng.uniform(0.5, 1.5)), (i, "Sz", -1, "I", 0.2 * rng.normal())]
    return sites, terms


def _spin_boson():
    # not self-adjoint: H^dagger differs from H
    return ([("spin", 2), ("boson", 5), ("spin", 3), ("spin", 2), ("spin", 2)],
            [(0, "Sy", 1, "N", 0.7), (2, "Sy", -1, "I", 0.4), (0, "Sm", 1, "adag", 0.5), (0, "Sp", 1, "a", 0.45),
             (2, "Sx", 0, "Sy", 0.3), (1, "N", -1, "I", 1.1), (3, "Sy", 4, "Sp", 0.25), (4, "Sy", -1, "I", -0.6)])


CASES = {
    "dm7": _dm(7, 2, 1),
    "dm_spin1_ring9": _dm(9, 3, 2, ring=True),     # 3^9 states: two low blocks of 3^8, ragged chunks
    "spin_boson": _spin_boson(),
    "dm_ring16": _dm(16, 2, 3, ring=True),          # 2^16 states: eight low blocks
}


def _scale(sites, terms, x, nvec, adjoint=False):
    H = abs(oracle.dense(sites, terms, sparse=True))
    if adjoint:
        H = H.T.tocsr()
    return np.asarray(H @ np.abs(x).reshape(-1, nvec)).reshape(-1)


def _close(got, ref, scale, tol, what):
    err = np.abs(got - ref)
    bad = np.flatnonzero(err > tol * scale + 1e-300)
    assert bad.size == 0, f"{what}: {bad.size} out of tolerance, worst {err[bad[:3]]} vs {scale[bad[:3]]}"


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cdt,tol", [("complex128", TOL_F64), ("complex64", TOL_F32)])
@pytest.mark.parametrize("nvec", [1, 2, 3])
def test_one_pass_equals_two_passes_and_matches_oracle(name, cdt, tol, nvec):
    torch = torch_cuda()
    sites, terms = CASES[name]
    h = _ham(sites, terms)
    xt = torch.from_numpy(_cx(h.D, 31 + nvec, nvec)).to("cuda", getattr(torch, cdt))
    xr = xt.cpu().numpy().astype(np.complex128)
    Hd = oracle.dense(sites, terms, sparse=True)
    for adj in (False, True):
        y1 = h.apply_ex(xt, transpose=adj)
        y2 = h.apply_ex(xt, transpose=adj, scalar=True)
        y3 = h.apply_ex(xt, transpose=adj)
        y4 = h.apply_ex(xt, transpose=adj, mb=True)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2), f"{name} {cdt} nvec={nvec} adjoint={adj}: one pass != two passes"
        assert torch.equal(y1, y3), "not reproducible"
        assert torch.equal(y1, y4), "register-capped one pass differs"
        M = Hd.conj().T.tocsr() if adj else Hd
        ref = np.asarray(M @ xr.reshape(h.D, nvec)).reshape(-1)
        _close(y1.cpu().numpy().astype(np.complex128), ref, _scale(sites, terms, xr, nvec, adj), tol,
               f"{name} {cdt} nvec={nvec} adjoint={adj}")
    # the default call (untuned: two passes) and the adjoint entry point give the same bits
    assert torch.equal(h.apply(xt), h.apply_ex(xt))
    gx, _ = h.adjoint(xt, want_gcoef=False)
    assert torch.equal(gx, h.apply_ex(xt, transpose=True))


@pytest.mark.parametrize("name", ["dm_spin1_ring9", "spin_boson"])
def test_native_f64_one_pass(name):
    torch = torch_cuda()
    sites, terms = CASES[name]
    h = _ham(sites, terms)
    xt = torch.from_numpy(_cx(h.D, 41, 2)).cuda()
    y1 = h.apply_ex(xt, native_f64=True)
    y2 = h.apply_ex(xt, native_f64=True, scalar=True)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    xr = xt.cpu().numpy()
    ref = oracle.apply(sites, terms, xr, nvec=2)
    _close(y1.cpu().numpy(), ref, _scale(sites, terms, xr, 2), TOL_F64, f"{name} native")


def _term_scale(sites, terms, x):
    """sum_t |c_t| |O_t| |x|: the error scale of any evaluation of a sum of
    term products. Terms that cancel (Sx Sy - Sy Sx on the S+ S+ channel)
    leave a rounding residue of about 1e-17 of their own magnitude in an
    evaluation that forms them separately (the row-wise oracle), which the
    merged |H| |x| does not cover once x spans hundreds of decades."""
    xs = np.abs(x)
    tot = np.zeros(xs.size)
    for t in terms:
        tot += abs(oracle.dense(sites, [t], sparse=True)) @ xs
    return tot


def test_inputs_outside_the_double_float_window():
    """Elements from 1e-300 to 1e+300 in mixed rows: the split flags them and
    the gated native FP64 one-pass launch gives the result, bit-identical to
    native FP64 throughout."""
    torch = torch_cuda()
    sites, terms = CASES["dm_spin1_ring9"]
    h = _ham(sites, terms)
    rng = np.random.default_rng(5)
    x = _cx(h.D, 43)
    x *= 10.0 ** rng.uniform(-300, 300, size=h.D)
    xt = torch.from_numpy(x).cuda()
    y = h.apply_ex(xt)
    yn = h.apply_ex(xt, native_f64=True)
    torch.cuda.synchronize()
    assert torch.equal(y, yn)
    assert torch.equal(h.apply(xt), yn)         # the two-pass form's gated fallback too
    ref = oracle.apply(sites, terms, x)
    _close(y.cpu().numpy(), ref, _term_scale(sites, terms, x), TOL_F64, "wide range")


def test_vectors_not_aligned_to_a_complex_element_take_two_passes():
    """x and y 8-byte aligned (not 16): hm_apply runs the two passes (same
    bits) even where the tuner chose the one-pass kernel, the explicit
    one-pass request is refused."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError, _capi as C
    sites, terms = CASES["dm7"]
    h = _ham(sites, terms)
    h.tune(1, torch.complex128)
    xc = torch.from_numpy(_cx(h.D, 47)).cuda()
    xb = torch.empty(2 * h.D + 1, dtype=torch.float64, device="cuda")
    xb[1:] = torch.view_as_real(xc).reshape(-1)
    yb = torch.full((2 * h.D + 1,), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = h._lib.hm_apply(h._h, xb[1:].data_ptr(), yb[1:].data_ptr(), 1, C.HM_C128, st)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.equal(yb[1:], torch.view_as_real(h.apply(xc)).reshape(-1))
    assert torch.isnan(yb[:1]).all()
    rc = h._lib.hm_apply_ex(h._h, xb[1:].data_ptr(), yb[1:].data_ptr(), 1, C.HM_C128, 0, 0, st)
    assert rc == C.HM_ERR_UNSUPPORTED


def test_tuned_choice_and_lanczos():
    """hm_tune on a complex H times the one-pass kernel against the two tuned
    passes and keeps the faster; either way the result matches the oracle,
    and the Lanczos ground state (one-pass applies) matches the dense one."""
    torch = torch_cuda()
    sites, terms = CASES["dm_ring16"]
    h = _ham(sites, terms)
    xt = torch.from_numpy(_cx(h.D, 53)).cuda()
    ref = oracle.apply(sites, terms, xt.cpu().numpy())
    h.tune(1, torch.complex128)
    cfg = h.tuned_config(1, torch.complex128)
    assert cfg["one_pass"] in (0, 1) and cfg["one_pass_capped"] <= cfg["one_pass"]
    y = h.apply(xt).cpu().numpy()
    _close(y, ref, _scale(sites, terms, xt.cpu().numpy(), 1), TOL_F64, "tuned")
    s7, t7 = CASES["dm7"]
    h7 = _ham(s7, t7)
    e_exact = np.linalg.eigvalsh(oracle.dense(s7, t7))[0]
    r = h7.lanczos(torch.from_numpy(_cx(h7.D, 59)).cuda(), 100, reorth=True)
    assert abs(r["e0"] - e_exact) < 1e-9 * abs(e_exact)
