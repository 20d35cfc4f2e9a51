"""Device Lanczos against dense diagonalisation and the FP64 oracle Lanczos;
Hellmann-Feynman gradients against finite differences."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import ham, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-10), (np.float32, 1e-5)])
def test_ring12_ground_state_energy(dtype, tol):
    torch = torch_cuda()
    m = W.heisenberg_ring(12)
    H = oracle.dense(m.sites, m.terms).real
    w, V = np.linalg.eigh(H)
    h = ham(m)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    v0 = torch.from_numpy(W.vector(4096, 1)).to("cuda", tdt)
    r = h.lanczos(v0, 100, reorth=True, ritz_vector=True)
    assert abs(r["e0"] - w[0]) <= tol * abs(w[0])
    psi = r["psi0"].double().cpu().numpy()
    assert abs(np.dot(psi, V[:, 0])) >= 1 - (1e-8 if dtype == np.float64 else 1e-4)


def test_lanczos_matches_oracle_lanczos_coefficients():
    """First alpha/beta of the device recurrence equal the FP64 oracle's."""
    torch = torch_cuda()
    m = W.ferrimagnet_chain(8)
    D = oracle.dimension(m.sites)
    v0 = W.vector(D, 3)
    a_ref, b_ref, e_ref, _ = oracle.lanczos(m.sites, m.terms, v0, 12)
    h = ham(m)
    r = h.lanczos(torch.from_numpy(v0).cuda(), 12, reorth=True)
    assert np.allclose(r["alpha"][:8], a_ref[:8], rtol=1e-10, atol=1e-12)
    assert np.allclose(r["beta"][:8], b_ref[:8], rtol=1e-10, atol=1e-12)


def test_lanczos_breakdown_small_space():
    torch = torch_cuda()
    m = W.heisenberg_ring(4)
    h = ham(m)
    v0 = torch.from_numpy(W.vector(16, 2)).cuda()
    r = h.lanczos(v0, 40, reorth=True)
    assert r["breakdown"] and r["steps"] <= 16
    assert abs(r["e0"] + 2.0) < 1e-10


def test_not_hermitian_rejected():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError, _capi as C, Hamiltonian
    h = Hamiltonian([("spin", 2), ("spin", 2)], [(0, "Sp", 1, "Sm", 1.0)])
    with pytest.raises(HmError) as e:
        h.lanczos(torch.ones(4, dtype=torch.float64, device="cuda"), 4)
    assert e.value.code == C.HM_ERR_NOT_HERMITIAN


def test_hellmann_feynman_gradients():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import lanczos_e0
    m = W.square_lattice_xxz(2, 4, seed=4)
    D = oracle.dimension(m.sites)
    h = ham(m)
    c = torch.tensor([t[4] for t in m.terms], dtype=torch.float64, requires_grad=True)
    v0 = torch.from_numpy(W.vector(D, 1)).cuda()
    E = lanczos_e0(h, c, v0, steps=120, reorth=True)
    E.backward()
    Edense = lambda cc: np.linalg.eigvalsh(oracle.dense(m.sites, m.terms, coefs=cc).real)[0]
    assert abs(E.item() - Edense(c.detach().numpy())) < 1e-9
    eps = 1e-5
    for t in range(0, len(m.terms), 2):
        cp = c.detach().numpy().copy()
        cp[t] += eps
        cm = c.detach().numpy().copy()
        cm[t] -= eps
        fd = (Edense(cp) - Edense(cm)) / (2 * eps)
        assert abs(fd - c.grad[t].item()) < 1e-6, t


def test_lanczos_ferrimagnet_full_size_matches_oracle():
    """The 6.05e7-state ferrimagnetic chain: the first alpha/beta of the FP64
    device recurrence against the FP64 oracle Lanczos on the same v0 (about a
    minute of oracle applies on the host cores)."""
    torch = torch_cuda()
    m = W.ferrimagnet_chain(20)
    D = oracle.dimension(m.sites)
    v0 = W.vector(D, 13)
    steps = 6
    a_ref, b_ref, _, _ = oracle.lanczos(m.sites, m.terms, v0, steps, nthreads=oracle.max_threads())
    h = ham(m)
    r = h.lanczos(torch.from_numpy(v0).cuda(), steps, reorth=True)
    assert np.allclose(r["alpha"][:steps], a_ref[:steps], rtol=1e-10, atol=1e-12), (r["alpha"], a_ref)
    assert np.allclose(r["beta"][:steps - 1], b_ref[:steps - 1], rtol=1e-10, atol=1e-12), (r["beta"], b_ref)


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-9), (np.float32, 2e-5)])
def test_lanczos_tavis_cummings_1e9_ground_state(dtype, tol):
    """200 Lanczos steps on the 1.07e9-state Tavis-Cummings model (24 spins,
    64 boson levels): E0 equals the vacuum energy -omega0 N / 2 = -12 (pinned
    on the CPU for small N); FP32 storage keeps FP64 dots."""
    torch = torch_cuda()
    m = W.tavis_cummings(24, 64, seed=7)
    h = ham(m)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    v0 = W.torch_vector(h.D, 11, dtype=tdt)
    r = h.lanczos(v0, 200)
    del v0
    torch.cuda.empty_cache()
    assert abs(r["e0"] + 12.0) <= tol * 12.0, r["e0"]


def test_hellmann_feynman_on_the_4x5_lattice():
    """Config-4 lattice (D = 2^20): Lanczos E0 with Hellmann-Feynman coupling
    gradients against central differences of the device Lanczos E0."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import lanczos_e0
    m = W.square_lattice_xxz(4, 5, seed=4)
    D = oracle.dimension(m.sites)
    h = ham(m)
    c0 = [t[4] for t in m.terms]
    v0 = torch.from_numpy(W.vector(D, 1)).cuda()
    c = torch.tensor(c0, dtype=torch.float64, requires_grad=True)
    E = lanczos_e0(h, c, v0, steps=150, reorth=True)
    E.backward()
    grad = c.grad.clone()

    def e0(cc):
        with torch.no_grad():
            return lanczos_e0(h, torch.tensor(cc, dtype=torch.float64), v0, steps=150, reorth=True).item()

    eps = 1e-4
    rng = np.random.default_rng(0)
    for t in sorted(rng.choice(len(c0), size=6, replace=False)):
        cp, cm = list(c0), list(c0)
        cp[t] += eps
        cm[t] -= eps
        fd = (e0(cp) - e0(cm)) / (2 * eps)
        assert abs(fd - grad[t].item()) < 1e-6 * max(1.0, abs(fd)), (t, fd, grad[t].item())
