"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle element by element."""
import numpy as np
import pytest

import oracle

TOL_F64 = 1e-12   # relative, FP64 storage
TOL_F32 = 1e-5    # relative, FP32 storage


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def ham(model):
    from paper_2606_02169_gb300 import Hamiltonian
    return Hamiltonian(model.sites, model.terms)


_ABS_CACHE = {}


def abs_matrix(model):
    key = (tuple(model.sites), tuple(model.terms))
    if key not in _ABS_CACHE:
        _ABS_CACHE.clear()
        _ABS_CACHE[key] = abs(oracle.dense(model.sites, model.terms, sparse=True))
    return _ABS_CACHE[key]


def abs_bound(model, x):
    """(|H| |x|)_F from the (sparse) Kronecker assembly: the natural per-row
    error scale of a sum of products."""
    H = abs_matrix(model)
    D = H.shape[0]
    nvec = x.size // D
    xs = np.abs(np.asarray(x, dtype=np.float64).reshape(D, nvec))
    return np.asarray(H @ xs).reshape(-1)


def abs_terms(model):
    """A term list whose operators have non-negative matrix elements that
    bound each term's |c_t| |O_t| elementwise: Sy -> Sx (|Sy| equals Sx
    elementwise), Sz on a spin-s site -> s I (|m| <= s, exact for s = 1/2);
    the other operators (Sx, S+-, Sz^2, S+-^2, N, a, adag, I) are
    non-negative already."""
    out = []
    for (i, oi, j, oj, c) in model.terms:
        f = abs(c)
        ops = []
        for site, op in ((i, oi), (j, oj)):
            if site >= 0:
                kind, d = model.sites[site]
                if op == "Sy":
                    op = "Sx"
                elif op == "Sz":
                    f *= (d - 1) / 2.0
                    op = "I"
            ops.append((site, op))
        out.append((ops[0][0], ops[0][1], ops[1][0], ops[1][1], f))
    return out


def row_abs_bound(model, x, rows):
    """sum_t |c_t| (|O_t| |x|)_F for the sampled rows F (an upper bound on the
    per-term error scale, from the row-wise oracle on |x|): the tolerance
    scale of sampled rows of vectors held on the host."""
    return np.abs(oracle.rows(model.sites, abs_terms(model), np.abs(np.asarray(x, dtype=np.float64)), rows).real)


def apply_abs_bound(model, x, nvec=1):
    """The same bound for every element of x (nvec right-hand sides), from
    the row-wise oracle's full apply on |x|."""
    xa = np.abs(np.asarray(x, dtype=np.float64))
    return np.abs(oracle.apply(model.sites, abs_terms(model), xa, nvec=nvec).real)


def row_scale_bound(model, xmax):
    """Crude per-row bound sum_t |c_t| max|O_t| * max|x| for sampled rows of
    systems too large to assemble."""
    def opmax(kind, d):   # bound on any local matrix element on that site
        if kind == "boson":
            return float(d - 1)                     # N = a^dag a reaches n_max
        s = (d - 1) / 2.0
        return (s + 1.0) ** 2                       # covers S+-, Sz^2, S+-^2
    tot = 0.0
    for (i, oi, j, oj, c) in model.terms:
        mi = opmax(*model.sites[i])
        mj = 1.0 if j < 0 else opmax(*model.sites[j])
        tot += abs(c) * mi * mj
    return tot * xmax


def check_close(got, ref, scale, tol, what=""):
    """Elementwise |got - ref| <= tol * scale (+ tiny) and normwise relative
    error <= tol. Returns (max elementwise ratio, normwise error)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref)
    assert np.abs(ref.imag).max(initial=0) < 1e-12 * (np.abs(ref).max(initial=0) + 1), "oracle gave imaginary y"
    ref = ref.real
    err = np.abs(got - ref)
    lim = tol * scale + 1e-300
    bad = np.flatnonzero(err > lim)
    nrm = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    assert bad.size == 0, (f"{what}: {bad.size} elements out of tolerance, worst at {bad[:5]}: "
                           f"got {got[bad[:5]]} ref {ref[bad[:5]]} scale {scale[bad[:5]]}")
    assert nrm <= tol, f"{what}: normwise error {nrm}"
    return float((err / (scale + 1e-300)).max(initial=0)), float(nrm)
