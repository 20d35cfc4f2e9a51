"""Pins of the sector oracle (oracle.sector_*, Sec. VI case 2, App. D) to
things other than itself: the App. D table and worked update (golden file),
combinatorial closed forms, brute-force enumeration, the full spectrum, and
the Jaynes-Cummings doublets of App. C."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "appendix_d_sector.txt")


def _golden():
    table, update = [], None
    for line in open(GOLD):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "table":
            table.append((f[1], int(f[2])))
        elif f[0] == "update":
            kv = dict(p.split("=") for p in f[1:])
            update = (tuple(int(s) for s in kv["sites"].split(",")), int(kv["target"]), int(kv["source"]))
    return table, update


def test_appendix_d_table():
    table, _ = _golden()
    sites = [("spin", 2)] * 4
    basis = oracle.sector_basis(sites, 2)          # 2 ups of 4 = zero magnetization
    assert [format(int(b), "04b") for b in basis] == [s for s, _ in table]
    for s, idx in table:
        digits = [int(c) for c in s]
        assert oracle.sector_rank([2] * 4, 2, digits) == idx
        assert oracle.sector_unrank([2] * 4, 2, idx) == digits


def test_appendix_d_worked_update():
    _, (sites_pm, tgt, src) = _golden()
    J = 1.3
    sites = [("spin", 2)] * 4
    i, j = sites_pm
    terms = [(i, "Sp", j, "Sm", J / 2)]
    x = np.zeros(6)
    x[src] = 1.0
    y = oracle.sector_apply(sites, terms, 2, x)
    want = np.zeros(6)
    want[tgt] = J / 2
    assert np.allclose(y, want, atol=1e-15)
    assert np.allclose(oracle.sector_rows(sites, terms, 2, x, list(range(6))), want, atol=1e-15)
    # a source outside the sector contributes nothing (failed lookup): a lone
    # S+ leaves the sector, so its restriction to the sector is zero
    assert np.allclose(oracle.sector_rows(sites, [(0, "Sp", -1, "I", 1.0)], 2, np.ones(6), list(range(6))), 0)


@pytest.mark.parametrize("n", [1, 4, 7, 10])
def test_spin_half_sector_dimension_is_binomial(n):
    for k in range(n + 1):
        assert oracle.sector_dimension([("spin", 2)] * n, k) == math.comb(n, k)


@pytest.mark.parametrize("dims", [[2] * 9, [3] * 6, [2, 4, 3, 2, 5]])
def test_sector_counts_by_enumeration(dims):
    """cnt[k][r] = number of digit tuples of sites k..N-1 summing to r, by
    brute-force enumeration of every suffix; for spins-1/2 it is C(N-k, r)."""
    import itertools
    total = sum(d - 1 for d in dims)
    cnt = oracle.sector_counts(dims, total)
    for k in range(len(dims) + 1):
        want = np.zeros(total + 1, dtype=np.int64)
        for tup in itertools.product(*[range(d) for d in dims[k:]]):
            want[sum(tup)] += 1
        assert list(cnt[k][: total + 1]) == list(want), k
        if all(d == 2 for d in dims):
            assert list(want) == [math.comb(len(dims) - k, r) for r in range(total + 1)]


def test_mixed_sector_dimensions_and_ranking_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(5):
        dims = [int(d) for d in rng.integers(2, 5, size=5)]
        sites = [("spin", d) for d in dims]
        D = oracle.dimension(sites)
        tot = 0
        for K in range(sum(d - 1 for d in dims) + 1):
            basis = oracle.sector_basis(sites, K)
            assert basis.size == oracle.sector_dimension(sites, K)
            tot += basis.size
            for r, I in enumerate(basis):
                digits = [int(v) for v in oracle.decode(dims, int(I))]
                assert oracle.sector_rank(dims, K, digits) == r
                assert oracle.sector_unrank(dims, K, r) == digits
        assert tot == D
    # spin-1 triple with total 3: coefficient of t^3 in (1 + t + t^2)^3
    assert oracle.sector_dimension([("spin", 3)] * 3, 3) == 7


def _conserving_model(dims, kinds, seed):
    rng = np.random.default_rng(seed)
    n = len(dims)
    terms = []
    for i in range(n):
        for j in range(i + 1, n):
            if kinds[i] == "spin" and kinds[j] == "spin":
                J, Jz = rng.uniform(-1, 1, 2)
                terms += [(i, "Sp", j, "Sm", J / 2), (i, "Sm", j, "Sp", J / 2), (i, "Sz", j, "Sz", Jz)]
            elif kinds[i] != kinds[j]:
                s, b = (i, j) if kinds[i] == "spin" else (j, i)
                g = rng.uniform(0.1, 1.0)
                terms += [(s, "Sm", b, "adag", g), (s, "Sp", b, "a", g)]
    for i in range(n):
        if kinds[i] == "spin":
            terms.append((i, "Sz", -1, "I", rng.uniform(-1, 1)))
            if dims[i] > 2:
                terms.append((i, "Sz2", -1, "I", rng.uniform(-1, 1)))
        else:
            terms.append((i, "N", -1, "I", rng.uniform(0.5, 1.5)))
    return [(k, d) for k, d in zip(kinds, dims)], terms


@pytest.mark.parametrize("dims,kinds", [((2, 3, 2, 4), ("spin",) * 4),
                                        ((3, 2, 5), ("spin", "spin", "boson")),
                                        ((4, 2, 2, 3), ("boson", "spin", "spin", "spin"))])
def test_sector_spectra_make_up_the_full_spectrum(dims, kinds):
    """A digit-sum-conserving H is block diagonal over the sectors: the union
    of the sector spectra is the full spectrum."""
    sites, terms = _conserving_model(dims, kinds, 3)
    H = oracle.dense(sites, terms)
    assert np.allclose(H, H.conj().T)
    full = np.sort(np.linalg.eigvalsh(H))
    parts = []
    for K in range(sum(d - 1 for d in dims) + 1):
        b = oracle.sector_basis(sites, K)
        Hs = np.stack([oracle.sector_apply(sites, terms, K, e) for e in np.eye(b.size)], axis=1)
        assert np.allclose(Hs, H[np.ix_(b, b)])
        parts.append(np.linalg.eigvalsh(Hs))
    assert np.allclose(np.sort(np.concatenate(parts)), full, atol=1e-12)


@pytest.mark.parametrize("dims,kinds", [((2, 3, 2, 4, 3), ("spin",) * 5),
                                        ((2, 2, 2, 6), ("spin", "spin", "spin", "boson"))])
def test_sector_rows_equals_projection(dims, kinds):
    sites, terms = _conserving_model(dims, kinds, 9)
    K = sum(d - 1 for d in dims) // 2
    n = oracle.sector_dimension(sites, K)
    x = W.vector(n, 4, nvec=2)
    ref = oracle.sector_apply(sites, terms, K, x, nvec=2)
    got = oracle.sector_rows(sites, terms, K, x, list(range(n)), nvec=2)
    assert np.allclose(got, ref, atol=1e-13)


def test_ring4_ground_state_lives_in_zero_magnetization():
    m = W.heisenberg_ring(4)
    b = oracle.sector_basis(m.sites, 2)
    Hs = np.stack([oracle.sector_apply(m.sites, m.terms, 2, e) for e in np.eye(b.size)], axis=1)
    assert abs(np.linalg.eigvalsh(Hs)[0] + 2.0) < 1e-12


@pytest.mark.parametrize("K", [1, 2, 5])
def test_jaynes_cummings_excitation_sector_is_a_doublet(K):
    """One spin-1/2 + a boson (App. C), resonant w = w0 = 1: the sector of K
    excitations holds |down, K> and |up, K-1>, with energies
    (K - 1/2) +- g sqrt(K) (the doublet of App. C with n = K - 1)."""
    g = 0.37
    sites = [("spin", 2), ("boson", 12)]
    terms = [(1, "N", -1, "I", 1.0), (0, "Sz", -1, "I", 1.0), (0, "Sm", 1, "adag", g), (0, "Sp", 1, "a", g)]
    b = oracle.sector_basis(sites, K)
    assert b.size == 2
    Hs = np.stack([oracle.sector_apply(sites, terms, K, e) for e in np.eye(2)], axis=1)
    w = np.linalg.eigvalsh(Hs)
    assert np.allclose(w, [(K - 0.5) - g * math.sqrt(K), (K - 0.5) + g * math.sqrt(K)], atol=1e-13)
