"""Pins for the CPU oracle: closed forms, invariants, library routines and
brute force. None of these compare the oracle with itself or with the CUDA
library; each catches a different plausible mistake (dropped term, wrong
sign or index, transposed operand, wrong ladder factor, wrong digit order)."""
import itertools
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def oracle_matrix(sites, terms):
    """Brute force: the C oracle applied to every unit vector gives H column by column."""
    D = oracle.dimension(sites)
    H = np.zeros((D, D), dtype=np.complex128)
    for k in range(D):
        e = np.zeros(D)
        e[k] = 1.0
        H[:, k] = oracle.apply(sites, terms, e)
    return H


def spectrum(sites, terms):
    H = oracle_matrix(sites, terms)
    assert np.allclose(H, H.conj().T, atol=1e-13)
    return np.sort(np.linalg.eigvalsh(H))


# ----------------------------------------------------------------------------
# Indexing (Sec. III)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(2, 3, 4, 5, 2, 7), (2,) * 9, (3, 3, 3), (64, 2, 2), (2, 2, 64)])
def test_encode_decode_matches_numpy_ravel(dims):
    D = int(np.prod(dims))
    m, Dc = oracle.multipliers(dims)
    assert Dc == D
    # place values equal numpy's C-order strides (site 0 most significant)
    strides = np.array(np.zeros(dims).strides) // 8
    assert list(m) == list(strides)
    for I in list(range(0, D, max(1, D // 997))) + [D - 1]:
        digits = oracle.decode(dims, I)
        assert tuple(digits) == tuple(np.unravel_index(I, dims))
        assert oracle.encode(dims, digits) == I == np.ravel_multi_index(tuple(digits), dims)


def test_paper_testbed_dimensions():
    """D = prod d_i reproduces the three dimensions printed in Sec. V."""
    want = {}
    with open(os.path.join(GOLDEN, "paper_testbeds.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, _, D = line.split()
            want[name] = int(D)
    assert oracle.dimension(W.paper_c1_chain().sites) == want["C1"]
    assert oracle.dimension(W.paper_c2_chain().sites) == want["C2"]
    assert oracle.dimension([("spin", 2)] * 25) == want["C3"]


# ----------------------------------------------------------------------------
# Local algebra of the dense assembly
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 8])
def test_spin_matrices_obey_su2(d):
    s = (d - 1) / 2
    L = lambda op: oracle.local_matrix("spin", d, op)
    sz, sp, sm, sx, sy = L("Sz"), L("Sp"), L("Sm"), L("Sx"), L("Sy")
    assert np.allclose(sp @ sm - sm @ sp, 2 * sz)
    assert np.allclose(sx @ sy - sy @ sx, 1j * sz)
    assert np.allclose(sx @ sx + sy @ sy + sz @ sz, s * (s + 1) * np.eye(d))
    assert np.allclose(np.linalg.eigvalsh(sx), np.arange(d) - s)
    # App. B identity Sx^2 - Sy^2 = (S+^2 + S-^2)/2
    assert np.allclose(sx @ sx - sy @ sy, (L("Sp2") + L("Sm2")) / 2)


def test_boson_matrices():
    d = 9
    a, ad, n = (oracle.local_matrix("boson", d, o) for o in ("a", "adag", "N"))
    comm = a @ ad - ad @ a
    assert np.allclose(np.diag(comm)[:-1], 1.0)       # [a, a^dag] = 1 below the cut
    assert np.isclose(comm[-1, -1], -(d - 1))          # truncation corner
    assert np.allclose(n, np.diag(np.arange(d)))


# ----------------------------------------------------------------------------
# Row-wise oracle == Kronecker assembly on random mixed systems
# ----------------------------------------------------------------------------

MIXED = [
    ((2, 3, 4), None),
    ((3, 2, 5, 2), None),
    ((2, 4, 6), ["spin", "boson", "spin"]),
    ((5, 2, 3, 2, 2), ["boson", "spin", "spin", "spin", "spin"]),
    ((2, 2, 2, 2, 2, 2, 2), None),
]


@pytest.mark.parametrize("dims,kinds", MIXED)
@pytest.mark.parametrize("seed", [0, 1])
def test_rowwise_equals_kronecker(dims, kinds, seed):
    m = W.random_model(list(dims), kinds, nterms=30, seed=seed)
    D = oracle.dimension(m.sites)
    H = oracle.dense(m.sites, m.terms)
    rng = np.random.default_rng(seed + 10)
    x = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    y = oracle.apply(m.sites, m.terms, x)
    ref = H @ x
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
    # sampled rows agree with the full apply
    r = rng.integers(0, D, size=17)
    assert np.allclose(oracle.rows(m.sites, m.terms, x, r), y[r], rtol=0, atol=1e-13)


def test_sy_single_site_is_imaginary():
    sites = [("spin", 3)]
    H = oracle_matrix(sites, [(0, "Sy", -1, "I", 1.0)])
    assert np.allclose(H.real, 0) and not np.allclose(H.imag, 0)


# ----------------------------------------------------------------------------
# Closed forms
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 8])
def test_zeeman_levels(d):
    s = (d - 1) / 2
    h = 0.73
    levels = h * (np.arange(d) - s)
    assert np.allclose(spectrum([("spin", d)], [(0, "Sz", -1, "I", h)]), levels)
    # rotation invariance: a transverse field has the same spectrum; pins
    # the ladder square roots of the S+ and S- rules (Sec. IV.A)
    assert np.allclose(spectrum([("spin", d)], [(0, "Sx", -1, "I", h)]), levels)
    assert np.allclose(spectrum([("spin", d)], [(0, "Sp", -1, "I", h / 2), (0, "Sm", -1, "I", h / 2)]),
                       levels)


@pytest.mark.parametrize("d1,d2", [(2, 2), (2, 3), (3, 3), (3, 4), (2, 5)])
def test_two_spin_heisenberg_multiplets(d1, d2):
    """J S1.S2 has E(S) = (J/2)[S(S+1) - s1(s1+1) - s2(s2+1)], degeneracy 2S+1."""
    J = 1.3
    s1, s2 = (d1 - 1) / 2, (d2 - 1) / 2
    want = []
    S = abs(s1 - s2)
    while S <= s1 + s2 + 1e-9:
        want += [J / 2 * (S * (S + 1) - s1 * (s1 + 1) - s2 * (s2 + 1))] * int(round(2 * S + 1))
        S += 1
    got = spectrum([("spin", d1), ("spin", d2)], W.heisenberg_bond(0, 1, J))
    assert np.allclose(got, np.sort(want))
    if d1 == d2 == 2:   # singlet -3J/4, triplet J/4
        assert np.isclose(got[0], -0.75 * J) and np.allclose(got[1:], 0.25 * J)


def test_two_site_ladder_form_equals_cartesian_form():
    """(S+S- + S-S+)/2 + SzSz equals SxSx + SySy + SzSz (same spectrum)."""
    sites = [("spin", 3), ("spin", 4)]
    ladder = [(0, "Sp", 1, "Sm", 0.5), (0, "Sm", 1, "Sp", 0.5), (0, "Sz", 1, "Sz", 1.0)]
    assert np.allclose(oracle_matrix(sites, ladder), oracle_matrix(sites, W.heisenberg_bond(0, 1, 1.0)))


def test_four_site_ring_ground_state():
    m = W.heisenberg_ring(4, J=1.0)
    assert np.isclose(spectrum(m.sites, m.terms)[0], -2.0)


@pytest.mark.parametrize("n", [6, 8])
def test_xx_chain_free_fermions(n):
    """Open XX chain J sum (SxSx + SySy): Jordan-Wigner gives free fermions with
    eps_k = J cos(k pi/(n+1)); the many-body levels are all subset sums."""
    J = 0.9
    terms = []
    for i in range(n - 1):
        terms += [(i, "Sx", i + 1, "Sx", J), (i, "Sy", i + 1, "Sy", J)]
    eps = J * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    want = np.sort([sum(c) for r in range(n + 1) for c in itertools.combinations(eps, r)])
    got = spectrum([("spin", 2)] * n, terms)
    assert np.allclose(got, want, atol=1e-12)


@pytest.mark.parametrize("D_,E_", [(1.0, 0.3), (-0.7, 0.2)])
def test_spin1_zero_field_splitting(D_, E_):
    """App. B: D[Sz^2 - s(s+1)/3] + E[Sx^2 - Sy^2] for s=1 has levels -2D/3, D/3 +- E."""
    terms = [(0, "Sz2", -1, "I", D_), (0, "I", -1, "I", -2 * D_ / 3),
             (0, "Sp2", -1, "I", E_ / 2), (0, "Sm2", -1, "I", E_ / 2)]
    got = spectrum([("spin", 3)], terms)
    assert np.allclose(got, np.sort([-2 * D_ / 3, D_ / 3 + E_, D_ / 3 - E_]))


@pytest.mark.parametrize("d", [4, 5, 6])
def test_higher_spin_zfs_against_matrix_products(d):
    """S+^2 and S-^2 channels (App. B q = +-2) equal the squared ladder matrices."""
    H = oracle_matrix([("spin", d)], [(0, "Sp2", -1, "I", 1.0)])
    sp = oracle_matrix([("spin", d)], [(0, "Sp", -1, "I", 1.0)])
    assert np.allclose(H, sp @ sp)
    H = oracle_matrix([("spin", d)], [(0, "Sm2", -1, "I", 1.0)])
    sm = oracle_matrix([("spin", d)], [(0, "Sm", -1, "I", 1.0)])
    assert np.allclose(H, sm @ sm)


@pytest.mark.parametrize("boson_first", [False, True])
@pytest.mark.parametrize("omega,omega0,g", [(1.0, 1.0, 0.1), (1.0, 1.4, 0.25)])
def test_jaynes_cummings_doublets(boson_first, omega, omega0, g):
    """App. C with one spin: ground -omega0/2, doublets
    omega(n+1/2) +- sqrt(Delta^2/4 + g^2 (n+1)), top unpaired omega n_max + omega0/2."""
    L = 8
    m = W.tavis_cummings(1, L, omega, omega0, boson_first=boson_first)
    b = m.meta["boson"]
    s = 1 - b
    terms = [(b, "N", -1, "I", omega), (s, "Sz", -1, "I", omega0),
             (b, "adag", s, "Sm", g), (b, "a", s, "Sp", g)]
    delta = omega0 - omega
    want = [-omega0 / 2, omega * (L - 1) + omega0 / 2]
    for n in range(L - 1):
        r = np.sqrt(delta ** 2 / 4 + g ** 2 * (n + 1))
        want += [omega * (n + 0.5) + r, omega * (n + 0.5) - r]
    assert np.allclose(spectrum(m.sites, terms), np.sort(want))


# ----------------------------------------------------------------------------
# Exact offsets (Sec. IV.B worked example S+_i S-_j: I = F - M_i + M_j)
# ----------------------------------------------------------------------------

def test_pair_offset_example():
    dims = (3, 2, 4, 5)
    sites = [("spin", d) for d in dims]
    strides = np.array(np.zeros(dims).strides) // 8     # numpy place values
    i, j = 0, 2
    target = (1, 0, 2, 3)                                # n_i > 0, n_j < d_j - 1
    F = np.ravel_multi_index(target, dims)
    I = F - strides[i] + strides[j]
    src = list(target)
    src[i] -= 1
    src[j] += 1
    assert I == np.ravel_multi_index(tuple(src), dims)
    e = np.zeros(int(np.prod(dims)))
    e[I] = 1.0
    y = oracle.apply(sites, [(i, "Sp", j, "Sm", 1.0)], e)
    nz = np.flatnonzero(np.abs(y) > 0)
    assert list(nz) == [F]
    sp_i = oracle.local_matrix("spin", dims[i], "Sp")
    sm_j = oracle.local_matrix("spin", dims[j], "Sm")
    assert np.isclose(y[F], sp_i[target[i], src[i]] * sm_j[target[j], src[j]])


# ----------------------------------------------------------------------------
# Invariants
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [3, 4, 5])
def test_hermiticity_of_hermitian_term_lists(seed):
    m = W.random_model([3, 2, 4, 2, 3], nterms=20, seed=seed, hermitian=True)
    D = oracle.dimension(m.sites)
    rng = np.random.default_rng(seed)
    x, y = rng.standard_normal(D), rng.standard_normal(D)
    lhs = np.vdot(y, oracle.apply(m.sites, m.terms, x))
    rhs = np.vdot(oracle.apply(m.sites, m.terms, y), x)
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1)


def _sector_vector(dims, Mtot, rng):
    D = int(np.prod(dims))
    x = np.zeros(D)
    for k in range(D):
        n = np.unravel_index(k, dims)
        m = sum(ni - (d - 1) / 2 for ni, d in zip(n, dims))
        if abs(m - Mtot) < 1e-9:
            x[k] = rng.standard_normal()
    return x


def test_total_sz_conservation_exact():
    dims = [2, 3, 2, 3, 2]
    m = W.xxz_spin1_chain(5)
    m = W.Model("mixed", [("spin", d) for d in dims], m.terms)
    rng = np.random.default_rng(9)
    x = _sector_vector(dims, 0.5, rng)
    y = oracle.apply(m.sites, m.terms, x).real
    outside = _sector_vector(dims, 0.5, np.random.default_rng(1)) == 0
    assert np.all(y[outside] == 0.0)       # exactly zero outside the sector
    assert np.linalg.norm(y) > 0


def test_tavis_cummings_excitation_number_conserved():
    m = W.tavis_cummings(3, 6, seed=11)
    dims = m.dims
    D = int(np.prod(dims))
    b = m.meta["boson"]
    def nexc(k):
        n = np.unravel_index(k, dims)
        return sum(n)    # boson occupation + number of up spins (digit 1 = up)
    rng = np.random.default_rng(2)
    x = np.array([rng.standard_normal() if nexc(k) == 3 else 0.0 for k in range(D)])
    y = oracle.apply(m.sites, m.terms, x).real
    mask = np.array([nexc(k) != 3 for k in range(D)])
    assert np.all(y[mask] == 0.0) and np.linalg.norm(y) > 0


# ----------------------------------------------------------------------------
# Lanczos and gradients
# ----------------------------------------------------------------------------

def test_lanczos_matches_dense_eigensolver_ring12():
    m = W.heisenberg_ring(12)
    D = 4096
    H = oracle.dense(m.sites, m.terms).real
    e_dense = np.linalg.eigvalsh(H)[0]
    v0 = W.vector(D, seed=1)
    _, _, e0, psi = oracle.lanczos(m.sites, m.terms, v0, 100)
    assert abs(e0 - e_dense) <= 1e-10 * abs(e_dense)
    r = H @ psi - e0 * psi
    assert np.linalg.norm(r) < 1e-6


def test_term_gradients_match_finite_differences():
    """L(c) = ||H(c) x - b||^2 is quadratic in c: central differences are
    exact up to rounding; dL/dc_t = Re <2(Hx - b)| O_t |x>."""
    m = W.square_lattice_xxz(2, 3, seed=4)
    D = oracle.dimension(m.sites)
    x, b = W.vector(D, 5), W.vector(D, 6)
    c0 = np.array([t[4] for t in m.terms])
    L = lambda c: float(np.linalg.norm(oracle.apply(m.sites, m.terms, x, coefs=c).real - b) ** 2)
    gy = 2 * (oracle.apply(m.sites, m.terms, x).real - b)
    g = oracle.term_gradients(m.sites, m.terms, gy, x).real
    h = 1e-6
    for t in range(len(c0)):
        e = np.zeros_like(c0)
        e[t] = h
        fd = (L(c0 + e) - L(c0 - e)) / (2 * h)
        assert abs(fd - g[t]) <= 1e-7 * max(1.0, abs(g[t]))


def test_hellmann_feynman_matches_finite_differences():
    m = W.square_lattice_xxz(2, 3, seed=4)
    c0 = np.array([t[4] for t in m.terms])
    E = lambda c: np.linalg.eigvalsh(oracle.dense(m.sites, m.terms, coefs=c).real)[0]
    w, V = np.linalg.eigh(oracle.dense(m.sites, m.terms).real)
    psi = V[:, 0]
    g = oracle.term_gradients(m.sites, m.terms, psi, psi).real
    h = 1e-5
    for t in range(len(c0)):
        e = np.zeros_like(c0)
        e[t] = h
        fd = (E(c0 + e) - E(c0 - e)) / (2 * h)
        assert abs(fd - g[t]) <= 1e-6


@pytest.mark.parametrize("nspins", [3, 4, 6])
def test_tavis_cummings_ground_state_is_the_vacuum(nspins):
    """Tavis-Cummings with omega = omega0 = 1 and g_i ~ U[0.05, 0.15] (the
    workload's draw): every coupling term annihilates |n=0, all spins down>,
    so it is an eigenstate of energy -omega0 N/2; with sqrt(sum g_i^2) < 1 no
    excitation sector reaches below it, so it is the ground state. Dense
    diagonalisation confirms E0 = -N/2 for small N (the reading behind the
    exact E0 = -12 of the 24-spin model), and that a coupling scaled past the
    threshold does move the ground state below the vacuum."""
    m = W.tavis_cummings(nspins, 16, seed=7)
    g = np.array(m.meta["g"])
    assert np.sqrt((g ** 2).sum()) < 1.0
    w = np.linalg.eigvalsh(oracle.dense(m.sites, m.terms).real)
    assert abs(w[0] + nspins / 2) < 1e-12
    assert w[1] > -nspins / 2 + 1.0 - np.sqrt((g ** 2).sum()) - 1e-9
    strong = [(i, oi, j, oj, c * (3.0 / np.sqrt((g ** 2).sum()) if oi in ("adag", "a") else 1.0))
              for (i, oi, j, oj, c) in m.terms]
    ws = np.linalg.eigvalsh(oracle.dense(m.sites, strong).real)
    assert ws[0] < -nspins / 2 - 0.1


def test_counter_based_inputs_match_published_splitmix64_outputs():
    """x_i is built from output i+1 of splitmix64 seeded with the seed:
    (z >> 11) * 2^-53 - 1/2. The oracle's generator reproduces the
    generator's published outputs (a wrong constant, shift or counter offset
    fails here), and its FP32 form is that value rounded to float."""
    rows = []
    with open(os.path.join(GOLDEN, "splitmix64_outputs.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                seed, k, z = (int(t) for t in line.split())
                rows.append((seed, k, z))
    assert len(rows) == 8
    for seed, k, z in rows:
        want = float(z >> 11) * 2.0 ** -53 - 0.5
        got = oracle.hashed_values(seed, np.array([k - 1]), False)[0]
        assert got == want, (seed, k)
        got32 = oracle.hashed_values(seed, np.array([k - 1]), True)[0]
        assert got32 == float(np.float32(want)), (seed, k)


def test_counter_based_inputs_agree_between_oracle_and_inputs_module():
    """The synthesised vector of the large sampled tests: the oracle's C
    generator and the inputs module's numpy generator (both written from the
    published splitmix64 definition) give the same values, and the oracle's
    rows with that vector equal its rows with the same vector passed in."""
    idx = np.concatenate([np.arange(1000), np.array([2 ** 31 - 1, 2 ** 31, 2 ** 32 + 7, 6_973_568_801])])
    for seed in (0, 21, 2 ** 63 + 5):
        for f32 in (False, True):
            assert np.array_equal(oracle.hashed_values(seed, idx, f32), W.hashed_values(seed, idx, f32))
    v = W.hashed_values(1, np.arange(100000))
    assert abs(v.mean()) < 0.01 and v.min() >= -0.5 and v.max() < 0.5
    m = W.random_model([3, 2, 4, 2, 3], None, nterms=20, seed=4)
    D = oracle.dimension(m.sites)
    x = W.hashed_values(9, np.arange(D), f32=True)
    rows = np.arange(0, D, 7)
    assert np.array_equal(oracle.rows_hashed(m.sites, m.terms, 9, rows, f32=True), oracle.rows(m.sites, m.terms, x, rows))
