"""Pins of oracle.evolve (y = exp(-i t H) x, hbar = 1) against closed forms
and invariants: a spin-1/2 Rabi rotation, spin-1 Larmor phases, the
Heisenberg dimer's singlet/triplet beat, a resonant Jaynes-Cummings pair
(App. C), unitarity, the group law, t = 0, the generator (-i H x as the
time derivative at t = 0, against the row-wise oracle) and a sector
restriction that equals the full-basis evolution of a state inside it."""
import numpy as np
import pytest

import oracle
import workloads as W


def test_rabi_rotation_of_one_spin_half():
    # H = Omega S_x; |up> is the digit n = 1 (n = m + s)
    Om, t = 1.7, 0.9
    y = oracle.evolve([("spin", 2)], [(0, "Sx", -1, "I", Om)], [0.0, 1.0], t)
    assert np.allclose(y, [-1j * np.sin(Om * t / 2), np.cos(Om * t / 2)], atol=1e-14)


def test_larmor_phases_of_spin_one():
    h, t = 0.6, 2.3
    x = np.array([0.2, -0.5, 0.7j])
    y = oracle.evolve([("spin", 3)], [(0, "Sz", -1, "I", h)], x, t)
    m = np.array([-1.0, 0.0, 1.0])
    assert np.allclose(y, np.exp(-1j * h * m * t) * x, atol=1e-14)


def test_heisenberg_dimer_singlet_triplet_beat():
    # H = J S1.S2: triplet J/4, singlet -3J/4. |up,down> (index 2) =
    # (|T0> + |S>)/sqrt 2 beats into |down,up> (index 1).
    J, t = 1.3, 0.77
    terms = [(0, "Sz", 1, "Sz", J), (0, "Sp", 1, "Sm", J / 2), (0, "Sm", 1, "Sp", J / 2)]
    x = np.zeros(4)
    x[2] = 1.0
    y = oracle.evolve([("spin", 2)] * 2, terms, x, t)
    a, b = np.exp(-1j * J * t / 4), np.exp(3j * J * t / 4)
    assert np.allclose(y, [0, (a - b) / 2, (a + b) / 2, 0], atol=1e-14)


def test_resonant_jaynes_cummings_pair():
    # H = g (a^dag S- + a S+) couples |up, 0> and |down, 1> with element g
    g, t = 0.8, 1.1
    sites = [("spin", 2), ("boson", 3)]
    terms = [(0, "Sm", 1, "adag", g), (0, "Sp", 1, "a", g)]
    up0 = oracle.encode([2, 3], [1, 0])
    dn1 = oracle.encode([2, 3], [0, 1])
    x = np.zeros(6)
    x[up0] = 1.0
    y = oracle.evolve(sites, terms, x, t)
    want = np.zeros(6, dtype=complex)
    want[up0], want[dn1] = np.cos(g * t), -1j * np.sin(g * t)
    assert np.allclose(y, want, atol=1e-14)


@pytest.fixture(scope="module")
def model():
    return W.random_model([2, 3, 2, 4], None, nterms=14, seed=5, hermitian=True)


def _cx(D, seed):
    return W.vector(D, seed) + 1j * W.vector(D, seed + 1)


def test_unitarity_group_law_and_identity(model):
    m = model
    D = oracle.dimension(m.sites)
    x = _cx(D, 3)
    y = oracle.evolve(m.sites, m.terms, x, 0.7)
    assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-13
    y2 = oracle.evolve(m.sites, m.terms, y, 0.5)
    assert np.allclose(y2, oracle.evolve(m.sites, m.terms, x, 1.2), atol=1e-13)
    assert np.allclose(oracle.evolve(m.sites, m.terms, x, 0.0), x, atol=1e-14)
    assert np.allclose(oracle.evolve(m.sites, m.terms, y, -0.7), x, atol=1e-13)


def test_generator_is_minus_i_h(model):
    """(y(d) - y(-d)) / 2d = -i H x + O(d^2 |H|^3 |x|), H x from the
    row-wise oracle (independent of the dense assembly)."""
    m = model
    D = oracle.dimension(m.sites)
    x = _cx(D, 9)
    d = 1e-4
    fd = (oracle.evolve(m.sites, m.terms, x, d) - oracle.evolve(m.sites, m.terms, x, -d)) / (2 * d)
    hx = oracle.apply(m.sites, m.terms, x)
    assert np.allclose(fd, -1j * hx, atol=1e-6 * np.abs(hx).max())


def test_sector_evolution_is_the_full_evolution_of_a_sector_state():
    sites = [("spin", 2)] * 6
    terms = []
    for i in range(6):
        j = (i + 1) % 6
        a, b = min(i, j), max(i, j)
        terms += [(a, "Sp", b, "Sm", 0.5), (a, "Sm", b, "Sp", 0.5), (a, "Sz", b, "Sz", 0.8)]
        terms.append((i, "Sz", -1, "I", 0.1 * i))
    bidx = oracle.sector_basis(sites, 3)
    xs = _cx(bidx.size, 4)
    full = np.zeros(2 ** 6, dtype=complex)
    full[bidx] = xs
    yf = oracle.evolve(sites, terms, full, 0.9)
    ys = oracle.evolve(sites, terms, xs, 0.9, sector_total=3)
    assert np.allclose(ys, yf[bidx], atol=1e-13)
    mask = np.ones(2 ** 6, dtype=bool)
    mask[bidx] = False
    assert np.abs(yf[mask]).max() < 1e-13
