"""Host logic of sector plans (hm_create_sector), on the CPU: the tables it
would upload (hm_plan_export bit 2, no GPU) run through a numpy emulation of
the sector kernel and are compared with the sector oracle's projection; and
the table shapes the kernel relies on (folded diagonal channels, rank-delta
tables for adjacent-site moves, 64-bit deltas for large sectors)."""
import numpy as np
import pytest

import oracle
import workloads as W
from plan_emulator import emulate_sector, emulate_sector_blk


@pytest.fixture(scope="module")
def capi():
    from paper_2606_02169_gb300 import build as B
    B.build()
    from paper_2606_02169_gb300 import _capi
    _capi.load()
    return _capi


def _sector(capi, sites, terms, total):
    return capi.plan_export(sites, terms, 4 | (total << 8))


def _conserving(dims, kinds, seed):
    rng = np.random.default_rng(seed)
    n = len(dims)
    terms = []
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < 0.6 and kinds[i] == "spin" and kinds[j] == "spin":
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
    terms.append((0, "I", -1, "I", 0.25))
    return [(k, d) for k, d in zip(kinds, dims)], terms


CASES = [((2, 3, 2, 4, 2), ("spin",) * 5, 4),
         ((3, 2, 5, 2), ("spin", "spin", "boson", "spin"), 3),
         ((6, 2, 2, 2, 2), ("boson", "spin", "spin", "spin", "spin"), 4),
         ((2,) * 10, ("spin",) * 10, 5),
         ((3,) * 7, ("spin",) * 7, 7)]


@pytest.mark.parametrize("dims,kinds,total", CASES)
@pytest.mark.parametrize("seed", [0, 1])
def test_sector_tables_reproduce_the_projection(capi, dims, kinds, total, seed):
    sites, terms = _conserving(dims, kinds, seed)
    S = _sector(capi, sites, terms, total)
    assert S["Dsec"] == oracle.sector_dimension(sites, total)
    for nvec in (1, 3):
        x = W.vector(S["Dsec"], 7 + seed, nvec=nvec)
        got = emulate_sector(S, x, nvec)
        ref = oracle.sector_apply(sites, terms, total, x, nvec=nvec)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def _ring(n, d=2, h=0.3, seed=0):
    rng = np.random.default_rng(seed)
    terms = []
    for i in range(n):
        j = (i + 1) % n
        a, b = min(i, j), max(i, j)
        terms += [(a, "Sp", b, "Sm", 0.5), (a, "Sm", b, "Sp", 0.5), (a, "Sz", b, "Sz", 1.0)]
        terms.append((i, "Sz", -1, "I", float(rng.uniform(-h, h))))
    return [("spin", d)] * n, terms


def test_ring_channels_fold_fields_and_tabulate_adjacent_moves(capi):
    """Periodic ring of 12 spins-1/2 with fields: the 12 field channels fold
    into the 12 bond-diagonal tables (listed first); the 22 moves on
    adjacent sites read a rank-delta table, the 2 moves of the closing bond
    (sites 0 and 11) are long moves summed over all sites while a row is
    unranked; no channel needs the rank tables; the result matches the
    oracle."""
    sites, terms = _ring(12)
    S = _sector(capi, sites, terms, 6)
    ch = S["ch"]
    diag = [c for c in ch if c[8]]
    hops = [c for c in ch if not c[8]]
    assert ch[:12] == diag
    assert len(diag) == 12 and all(c[5] >= 0 for c in diag)
    assert len(hops) == 24
    assert sum(c[1] >= 0 for c in hops) == 22
    assert all(c[1] <= -2 for c in hops if (c[4], c[5]) == (0, 11))
    assert len(S["lt"]) == 2 * 12 * 7 * 2          # 2 moves x 12 sites x (K + 1) totals x 2 digits
    assert not S["needA"] and not S["wide"]
    x = W.vector(S["Dsec"], 3)
    ref = oracle.sector_apply(sites, terms, 6, x)
    assert np.allclose(emulate_sector(S, x), ref, rtol=0, atol=1e-12)


def test_long_moves_beyond_the_table_budget_use_the_rank_tables(capi):
    """Many long moves on 16 sites: those whose per-site tables fit the
    budget read them, the rest update the rank from the rank tables; both
    agree with the oracle."""
    n = 16
    sites = [("spin", 2)] * n
    terms = []
    for a in range(n):
        for b in range(a + 2, n, 3):
            terms += [(a, "Sp", b, "Sm", 0.3 + 0.01 * (a + b)), (a, "Sm", b, "Sp", 0.3 + 0.01 * (a + b))]
    terms += [(k, "Sz", -1, "I", 0.1 * k) for k in range(n)]
    S = _sector(capi, sites, terms, 8)
    hops = [c for c in S["ch"] if not c[8]]
    assert any(c[1] <= -2 for c in hops) and any(c[1] == -1 for c in hops) and S["needA"]
    x = W.vector(S["Dsec"], 6)
    assert np.allclose(emulate_sector(S, x), oracle.sector_apply(sites, terms, 8, x), rtol=0, atol=1e-12)


def test_open_chain_needs_no_rank_tables(capi):
    sites, terms = _ring(10)
    terms = [t for t in terms if not (t[0] == 0 and t[2] == 9)]
    S = _sector(capi, sites, terms, 5)
    assert not S["needA"]
    x = W.vector(S["Dsec"], 4, nvec=2)
    ref = oracle.sector_apply(sites, terms, 5, x, nvec=2)
    assert np.allclose(emulate_sector(S, x, 2), ref, rtol=0, atol=1e-12)


def test_large_sectors_store_64_bit_deltas(capi):
    """C(40, 20) > 2^31 retained states: rank deltas are 64-bit; the
    tabulated delta of one adjacent move equals the difference of the two
    states' ranks (oracle.sector_rank)."""
    import math
    sites, terms = _ring(40, h=0.0)
    S = _sector(capi, sites, terms, 20)
    assert S["Dsec"] == math.comb(40, 20) and S["wide"]
    # target: digits 0..19 = 1, 20..39 = 0, hop S+_19 S-_20 seen from the
    # target with n_19 = 0, n_20 = 1 (the source has them swapped)
    tgt = [1] * 19 + [0, 1] + [0] * 19
    src = [1] * 20 + [0] * 20
    ch = [c for c in S["ch"] if (c[4], c[5]) == (19, 20) and not c[8] and c[6] == -1]
    assert len(ch) == 1 and ch[0][1] >= 0
    tb, dtab, rstride, dj = ch[0][:4]
    rem19 = 20 - sum(tgt[:19])
    delta = S["dl"][dtab + rem19 * rstride + tgt[19] * dj + tgt[20]]
    dims = [2] * 40
    assert delta == oracle.sector_rank(dims, 20, src) - oracle.sector_rank(dims, 20, tgt)


@pytest.mark.parametrize("K", [0, 1, 3, 6])
def test_tavis_cummings_excitation_sectors_with_capped_boson_digits(capi, K):
    """Five spins-1/2 coupled to one boson of 9 levels (more levels than the
    excitation number allows, so the rank tables cap the boson's digits at
    K + 1): every spin-boson move is long except the last spin's, and the
    tables reproduce the oracle's projection."""
    n = 5
    sites = [("spin", 2)] * n + [("boson", 9)]
    b = n
    terms = [(b, "N", -1, "I", 1.0)]
    for i in range(n):
        g = 0.1 + 0.03 * i
        terms += [(i, "Sz", -1, "I", 1.0 + 0.05 * i), (i, "Sp", b, "a", g), (i, "Sm", b, "adag", g)]
    S = _sector(capi, sites, terms, K)
    assert S["Dsec"] == oracle.sector_dimension(sites, K)
    assert S["d"][b] == min(9, K + 1)
    x = W.vector(S["Dsec"], 13)
    ref = oracle.sector_apply(sites, terms, K, x)
    assert np.allclose(emulate_sector(S, x), ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


BLK_CASES = [
    ((2,) * 15, ("spin",) * 15, 7),                                  # one prefix site
    ((2,) * 16, ("spin",) * 16, 5),                                  # two prefix sites
    ((6,) + (2,) * 12, ("boson",) + ("spin",) * 12, 6),              # boson prefix
    ((3, 2) + (2,) * 10 + (5,), ("spin",) * 12 + ("boson",), 7),     # boson in the suffix
    ((3, 3, 3, 3, 3, 3, 3, 3, 3, 3), ("spin",) * 10, 10),            # spin-1, 3^10 states
]


@pytest.mark.parametrize("dims,kinds,total", BLK_CASES)
def test_block_form_tables_reproduce_the_projection(capi, dims, kinds, total):
    """The block form's tables (hm_plan_export bits 2 and 4) run through the
    numpy emulation of its kernel equal the sector oracle's projection P H
    P^T x; the suffix sectors partition the suffix tuples, the blocks the
    retained states."""
    sites, terms = _conserving(dims, kinds, 12)
    B = capi.plan_export(sites, terms, 4 | 16 | (total << 8))
    assert B["ok"]
    n = oracle.sector_dimension(sites, total)
    x = W.vector(n, 3)
    ref = oracle.sector_apply(sites, terms, total, x)
    got = emulate_sector_blk(B, x)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    # structure: suffix sectors cover the suffix tuples, blocks the sector
    suffix_dims = [d for _, d in sites[B["h"]:]]
    assert B["off"][-1] == B["G"] == sum(oracle.sector_dimension([("spin", d) for d in suffix_dims], t)
                                         for t in range(total + 1))
    sizes = []
    for b in B["vb"]:
        P = sum((b // B["mp"][k]) % B["pdim"][k] for k in range(B["h"]))
        sizes.append(B["off"][total - P + 1] - B["off"][total - P])
    assert sum(sizes) == n
    assert [B["start"][b] for b in B["vb"]] == list(np.concatenate([[0], np.cumsum(sizes)[:-1]]))
    kinds_seen = {c[0] for c in B["ch"]}
    if B["h"] >= 2:
        assert kinds_seen >= {0, 1, 2, 3}      # prefix diagonal and moves, coupled diagonal and moves


def test_block_form_with_several_right_hand_sides(capi):
    sites, terms = _conserving((2,) * 15, ("spin",) * 15, 13)
    B = capi.plan_export(sites, terms, 4 | 16 | (6 << 8))
    n = oracle.sector_dimension(sites, 6)
    x = W.vector(n, 4, nvec=3)
    assert np.allclose(emulate_sector_blk(B, x, 3), oracle.sector_apply(sites, terms, 6, x, nvec=3),
                       rtol=0, atol=1e-12)


def test_block_form_rejections(capi):
    from paper_2606_02169_gb300._capi import HmError
    sites = [("spin", 2)] * 16
    with pytest.raises(HmError):       # empty sector
        capi.plan_export(sites, [(0, "Sz", -1, "I", 1.0)], 4 | 16 | (17 << 8))
    with pytest.raises(HmError):       # a lone Sx moves the digit sum
        capi.plan_export(sites, [(0, "Sx", -1, "I", 1.0)], 4 | 16 | (8 << 8))
