"""The one-spin case of the Tavis-Cummings workload (App. C, 64 boson
levels, the truncation of the 2^30-state benchmark) against the
Jaynes-Cummings closed form, with no oracle in between: H applied on the
GPU to the identity (nvec = D right-hand sides through the C ABI) gives H
column by column, and its spectrum is the ground level -omega0/2, the
unpaired top level omega n_max + omega0/2 and the doublets
omega (n + 1/2) +- sqrt(Delta^2 / 4 + g^2 (n + 1)), Delta = omega0 - omega."""
import numpy as np
import pytest

import workloads as W
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

L = 64


def _closed_form(omega, omega0, g):
    delta = omega0 - omega
    want = [-omega0 / 2, omega * (L - 1) + omega0 / 2]
    for n in range(L - 1):
        r = np.sqrt(delta ** 2 / 4 + g ** 2 * (n + 1))
        want += [omega * (n + 0.5) + r, omega * (n + 0.5) - r]
    return np.sort(want)


@pytest.mark.parametrize("boson_first", [False, True])
@pytest.mark.parametrize("omega,omega0,g", [(1.0, 1.0, 0.1), (1.0, 1.4, 0.25), (0.8, 1.1, 0.13)])
@pytest.mark.parametrize("dtype,tol", [("float64", 1e-11), ("float32", 2e-4)])
def test_jaynes_cummings_spectrum_on_the_gpu(boson_first, omega, omega0, g, dtype, tol):
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian
    m = W.tavis_cummings(1, L, omega, omega0, boson_first=boson_first)
    b = m.meta["boson"]
    s = 1 - b
    terms = [(b, "N", -1, "I", omega), (s, "Sz", -1, "I", omega0),
             (b, "adag", s, "Sm", g), (b, "a", s, "Sp", g)]
    h = Hamiltonian(m.sites, terms)
    D = h.D
    assert D == 2 * L
    eye = torch.eye(D, dtype=getattr(torch, dtype), device="cuda").reshape(-1)   # x[k*D + v] = delta_kv
    Hm = h.apply(eye).reshape(D, D).double().cpu().numpy()                         # row k, column v = H_kv
    assert np.abs(Hm - Hm.T).max() <= tol * 100           # Hermitian (real symmetric)
    ev = np.linalg.eigvalsh(0.5 * (Hm + Hm.T))
    want = _closed_form(omega, omega0, g)
    assert np.abs(ev - want).max() <= tol * np.abs(want).max(), (np.abs(ev - want).max(), dtype)
    # the excitation number n_b + (m + 1/2) is conserved: no element couples
    # different totals (digits: spin n = m + 1/2, boson n = occupation)
    k = np.arange(D)
    nb, ns = (k // 2, k % 2) if boson_first else (k % L, k // L)
    exc = nb + ns
    assert np.all(Hm[exc[:, None] != exc[None, :]] == 0.0)
