"""GPU parity of the adjoint pass: gx = H^T gy and the per-term coupling
gradients g_t = <gy| O_t |x>, against the oracle; and the autograd wrappers
against central finite differences."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu


def _transpose_model(m):
    """Oracle side of H^T: the dense transpose applied to gy."""
    return oracle.dense(m.sites, m.terms, sparse=True).T.tocsr()


@pytest.mark.parametrize("dims,kinds,seed", [
    ((3, 2, 4, 2, 3), None, 0),
    ((3, 2, 5, 2, 3, 4, 2, 3, 2), None, 1),
    ((2, 2, 2, 2, 2, 2, 2, 64), ["spin"] * 7 + ["boson"], 2),
    ((64, 2, 2, 2, 2, 2, 2, 2), ["boson"] + ["spin"] * 7, 3),
])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_adjoint_matches_oracle(dims, kinds, seed, dtype):
    torch = torch_cuda()
    m = W.random_model(list(dims), kinds, nterms=24, seed=seed)   # not Hermitian in general
    D = oracle.dimension(m.sites)
    gy = W.vector(D, seed + 1).astype(dtype).astype(np.float64)
    x = W.vector(D, seed + 2).astype(dtype).astype(np.float64)
    h = ham(m)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    gx, gc = h.adjoint(torch.from_numpy(gy).to("cuda", tdt), torch.from_numpy(x).to("cuda", tdt))
    torch.cuda.synchronize()
    HT = _transpose_model(m)
    ref = HT @ gy
    scale = np.asarray(abs(HT) @ np.abs(gy)).reshape(-1)
    tol = TOL_F64 if dtype == np.float64 else TOL_F32
    check_close(gx.double().cpu().numpy(), ref, scale, tol, "gx")
    gref = oracle.term_gradients(m.sites, m.terms, gy, x)
    gscale = np.array([np.vdot(np.abs(gy), np.abs(oracle.apply(m.sites, [(t[0], t[1], t[2], t[3], 1.0)], x)))
                       for t in m.terms]) + 1e-30
    # FP64 accumulation of the gradient in both cases; FP32 inputs are exact in FP64
    check_close(gc.cpu().numpy(), gref, np.maximum(gscale, 1e-12), 1e-11, "gcoef")


def test_dot_identity_nonhermitian():
    """<gy, H x> = <H^T gy, x> for a non-Hermitian list (H^T differs from H)."""
    torch = torch_cuda()
    m = W.random_model([3, 2, 4, 3, 2], None, nterms=30, seed=8)
    h = ham(m)
    x = torch.from_numpy(W.vector(h.D, 1)).cuda()
    gy = torch.from_numpy(W.vector(h.D, 2)).cuda()
    lhs = torch.dot(gy, h.apply(x)).item()
    gx, _ = h.adjoint(gy, x, want_gcoef=False)
    rhs = torch.dot(gx, x).item()
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_gradients_with_multiple_rhs():
    torch = torch_cuda()
    m = W.random_model([3, 2, 4, 2], None, nterms=16, seed=4)
    D = oracle.dimension(m.sites)
    nvec = 3
    gy = W.vector(D, 5, nvec=nvec)
    x = W.vector(D, 6, nvec=nvec)
    h = ham(m)
    _, gc = h.adjoint(torch.from_numpy(gy).cuda(), torch.from_numpy(x).cuda(), want_gx=False)
    ref = np.zeros(len(m.terms), dtype=np.complex128)
    for v in range(nvec):
        ref += oracle.term_gradients(m.sites, m.terms, gy.reshape(D, nvec)[:, v].copy(),
                                     x.reshape(D, nvec)[:, v].copy())
    assert np.allclose(gc.cpu().numpy(), ref.real, rtol=1e-11, atol=1e-12)


def _lattice_loss_setup(rows, cols):
    torch = torch_cuda()
    m = W.square_lattice_xxz(rows, cols, seed=4)
    D = oracle.dimension(m.sites)
    x = torch.from_numpy(W.vector(D, 5)).cuda()
    b = torch.from_numpy(W.vector(D, 6)).cuda()
    J = torch.tensor(m.meta["Jv"], dtype=torch.float64, requires_grad=True)
    Dl = torch.tensor(m.meta["Deltav"], dtype=torch.float64, requires_grad=True)
    hf = torch.tensor(m.meta["hv"], dtype=torch.float64, requires_grad=True)
    return m, x, b, J, Dl, hf


def _coefs(m, J, Dl, hf):
    import torch
    parts = []
    for bidx in range(len(m.meta["bonds"])):
        parts += [J[bidx], J[bidx], J[bidx] * Dl[bidx]]
    parts += [hf[i] for i in range(len(m.meta["hv"]))]
    return torch.stack(parts)


def test_residual_loss_gradients_vs_finite_differences():
    """L = ||H x - b||^2 on a 3x4 lattice: dL/dx, dL/dJ, dL/dDelta, dL/dh from
    the adjoint kernel vs central differences (step 1e-6) of the same GPU loss."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import hamiltonian_apply
    m, x, b, J, Dl, hf = _lattice_loss_setup(3, 4)
    h = ham(m)
    xr = x.clone().requires_grad_(True)

    def loss(J_, D_, h_, x_):
        y = hamiltonian_apply(h, _coefs(m, J_, D_, h_), x_)
        return ((y - b) ** 2).sum()

    L = loss(J, Dl, hf, xr)
    L.backward()
    eps = 1e-6
    with torch.no_grad():
        for name, P in (("J", J), ("Delta", Dl), ("h", hf)):
            for k in range(0, P.numel(), 3):
                old = P[k].item()
                P[k] = old + eps
                lp = loss(J, Dl, hf, x).item()
                P[k] = old - eps
                lm = loss(J, Dl, hf, x).item()
                P[k] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - P.grad[k].item()) <= 1e-6 * max(1.0, abs(fd)), (name, k)
        idx = np.random.default_rng(0).integers(0, x.numel(), size=20)
        for k in idx:
            e = torch.zeros_like(x)
            e[k] = eps
            fd = (loss(J, Dl, hf, x + e).item() - loss(J, Dl, hf, x - e).item()) / (2 * eps)
            assert abs(fd - xr.grad[k].item()) <= 1e-6 * max(1.0, abs(fd))


def test_residual_loss_gradients_vs_oracle_4x5():
    """Full-size 4x5 lattice (D = 2^20): coupling gradients of ||Hx - b||^2
    equal the oracle's <2(Hx-b)| O_t |x> assembled through the same chain rule."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import hamiltonian_apply
    m, x, b, J, Dl, hf = _lattice_loss_setup(4, 5)
    h = ham(m)
    y = hamiltonian_apply(h, _coefs(m, J, Dl, hf), x)
    L = ((y - b) ** 2).sum()
    L.backward()
    xn, bn = x.cpu().numpy(), b.cpu().numpy()
    gy = 2 * (oracle.apply(m.sites, m.terms, xn).real - bn)
    gt = oracle.term_gradients(m.sites, m.terms, gy, xn).real
    nb = len(m.meta["bonds"])
    Jv, Dv = np.array(m.meta["Jv"]), np.array(m.meta["Deltav"])
    gJ = np.array([gt[3 * k] + gt[3 * k + 1] + Dv[k] * gt[3 * k + 2] for k in range(nb)])
    gD = np.array([Jv[k] * gt[3 * k + 2] for k in range(nb)])
    gh = gt[3 * nb:]
    for got, ref in ((J.grad, gJ), (Dl.grad, gD), (hf.grad, gh)):
        assert np.allclose(got.numpy(), ref, rtol=1e-9, atol=1e-10)


def test_autograd_coefficient_sync_only_when_changed():
    """The autograd wrapper re-plans only when the coefficient tensor is a
    different tensor or was modified in place; an unchanged tensor skips the
    host read. A direct set_coefficients between calls is honoured."""
    torch = torch_cuda()
    from paper_2606_02169_gb300.autograd import hamiltonian_apply
    m = W.heisenberg_ring(8)
    h = ham(m)
    x = torch.from_numpy(W.vector(h.D, 3)).cuda()
    coefs = torch.tensor([t[4] for t in m.terms], dtype=torch.float64, device="cuda")
    reads = []
    orig = h.set_coefficients
    h.set_coefficients = lambda c: (reads.append(1), orig(c))[1]
    y0 = hamiltonian_apply(h, coefs, x)
    y1 = hamiltonian_apply(h, coefs, x)           # same tensor, unchanged: no re-plan
    assert torch.equal(y0, y1) and len(reads) == 0
    with torch.no_grad():
        coefs.mul_(2.0)                           # in place: version bump, re-plan
    y2 = hamiltonian_apply(h, coefs, x)
    assert len(reads) == 1 and torch.allclose(y2, 2 * y0, rtol=1e-13, atol=0)
    orig([t[4] for t in m.terms])                 # direct update back to the original
    y3 = hamiltonian_apply(h, coefs, x)           # must re-sync to 2x
    assert len(reads) == 2 and torch.allclose(y3, 2 * y0, rtol=1e-13, atol=0)
