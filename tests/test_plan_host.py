"""Host logic of the plan builder, on the CPU: the tables hm_create would
upload (hm_plan_export, no GPU) are run through a numpy emulation of the
kernel's per-block algorithm and compared with the oracle's Kronecker
assembly, for H and H^T."""
import numpy as np
import pytest

import oracle
import workloads as W
from plan_emulator import emulate


@pytest.fixture(scope="module")
def capi():
    from paper_2606_02169_gb300 import build as B
    B.build()
    from paper_2606_02169_gb300 import _capi
    _capi.load()
    return _capi


CASES = [
    ((3, 2, 4, 2, 3), None),
    ((3, 2, 5, 2, 3, 4, 2, 3, 2), None),
    ((2,) * 14, None),
    ((64, 2, 2, 2, 2, 2, 2, 2), ["boson"] + ["spin"] * 7),
    ((2, 2, 2, 2, 2, 2, 2, 64), ["spin"] * 7 + ["boson"]),
    ((3, 5, 2, 7, 3, 2, 2, 3), ["spin", "boson", "spin", "boson", "spin", "spin", "spin", "spin"]),
]


@pytest.mark.parametrize("dims,kinds", CASES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plan_tables_reproduce_h_and_transpose(capi, dims, kinds, seed):
    m = W.random_model(list(dims), kinds, nterms=24, seed=seed)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 7)
    H = oracle.dense(m.sites, m.terms, sparse=True)
    for which, M in ((0, H), (1, H.T)):
        P = capi.plan_export(m.sites, m.terms, which)
        y = emulate(P, x)
        ref = np.asarray(M @ x).real
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref), (which, P["nhigh"])


def test_imaginary_factors_with_real_product(capi):
    """SySy across the high/low split: each factor imaginary, product real."""
    sites = [("spin", d) for d in (3, 2, 5, 2, 3, 4, 2, 3, 2)]
    terms = [(3, "Sy", 0, "Sy", 0.37), (0, "Sy", 8, "Sy", -0.2)]
    D = oracle.dimension(sites)
    x = W.vector(D, 1)
    P = capi.plan_export(sites, terms, 0)
    assert P["nhigh"] >= 1
    ref = (oracle.dense(sites, terms, sparse=True) @ x).real
    assert np.allclose(emulate(P, x), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("dims,kinds", CASES[:4] + CASES[5:])
@pytest.mark.parametrize("seed", [3, 4])
def test_complex_h_as_two_real_plans(capi, dims, kinds, seed):
    """A term list with imaginary matrix elements (Sy factors): the exported
    real-part plan (which = 0) and imaginary-part plan (bit 3) give
    H = H_re + i H_im, and their transposes (bit 0) give H^T, against the
    oracle's complex Kronecker assembly."""
    m = W.random_model(list(dims), kinds, nterms=20, seed=seed)
    spins = [k for k, (kind, _) in enumerate(m.sites) if kind in ("spin", 0)]
    a, b = spins[0], spins[-1]
    terms = m.terms + [(a, "Sy", -1, "I", 0.6), (a, "Sx", b, "Sy", -0.4), (b, "Sy", a, "Sz", 0.3),
                       (b, "Sy", -1, "I", -0.2 * seed)]
    m = W.Model(m.name + "+Sy", m.sites, terms)
    D = oracle.dimension(m.sites)
    H = oracle.dense(m.sites, m.terms, sparse=True)
    assert abs(H.imag).max() > 0
    x = W.vector(D, 7) + 1j * W.vector(D, 8)
    for tr, M in ((0, H), (1, H.T)):
        Pr = capi.plan_export(m.sites, m.terms, tr)
        Pi = capi.plan_export(m.sites, m.terms, tr | 8)
        y = (emulate(Pr, x.real) - emulate(Pi, x.imag)) + 1j * (emulate(Pr, x.imag) + emulate(Pi, x.real))
        ref = np.asarray(M @ x)
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref), tr


def test_workload_plans(capi):
    """Split and channel structure of the workload shapes."""
    P = capi.plan_export(*_m(W.tavis_cummings(24, 64, seed=7)))
    assert P["B"] == 8192 and P["nblk"] == 2 ** 17 and P["nhigh"] == 17
    # boson last: every JC hop of a high spin is factorised into two groups
    # (a^dag S-: sqrt(n_b); a S+: sqrt(n_b+1)) with 17 members each
    off = P["grp"][P["n_grp_diag"]:]
    assert len(off) == 2 and all(g[3] - g[2] == 17 for g in off)
    P = capi.plan_export(*_m(W.ferrimagnet_chain(20)))
    assert P["B"] == 7776 and P["hermitian"]
    P = capi.plan_export(*_m(W.heisenberg_ring(12)))
    assert P["B"] == 4096 and P["nblk"] == 1


def _m(model):
    return model.sites, model.terms


@pytest.mark.parametrize("model", [W.ferrimagnet_chain(10), W.tavis_cummings(6, 8, seed=1),
                                   W.square_lattice_xxz(3, 4, seed=4), W.heisenberg_ring(13)])
def test_workload_shapes_small(capi, model):
    D = oracle.dimension(model.sites)
    x = W.vector(D, 2)
    P = capi.plan_export(model.sites, model.terms, 0)
    ref = oracle.apply(model.sites, model.terms, x).real
    assert np.linalg.norm(emulate(P, x) - ref) <= 1e-13 * np.linalg.norm(ref)


# ---- tile form (leaf-tiled kernel) -------------------------------------------------

TILE_CASES = CASES + [
    ((2,) * 12, None),
    ((2, 3) * 5, None),
    ((3,) * 9, None),
    ((5, 4, 3, 6, 2, 2), None),
    ((2,) * 6 + (64,), ["spin"] * 6 + ["boson"]),
]


@pytest.mark.parametrize("dims,kinds", TILE_CASES)
@pytest.mark.parametrize("nvec", [1, 3])
def test_tile_tables_reproduce_h_and_transpose(capi, dims, kinds, nvec):
    from plan_emulator import emulate_tile
    m = W.random_model(list(dims), kinds, nterms=24, seed=5)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 9, nvec=nvec)
    for which in (0, 1):
        try:
            T = capi.plan_export(m.sites, m.terms, which | 2 | (nvec << 8))
        except capi.HmError as e:
            assert e.code == capi.HM_ERR_UNSUPPORTED
            continue
        assert T["F"] * nvec <= 512 and T["nblk"] * T["R"] * T["F"] == D
        y = emulate_tile(T, x)
        ref = oracle.apply(m.sites, m.terms, x, nvec=nvec).real if which == 0 else \
            np.asarray(oracle.dense(m.sites, m.terms, sparse=True).T @ x.reshape(D, nvec)).real.reshape(-1)
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref), (which, T["F"], T["R"])


@pytest.mark.parametrize("model", [W.ferrimagnet_chain(12), W.tavis_cummings(6, 8, seed=1),
                                   W.square_lattice_xxz(3, 4, seed=4), W.heisenberg_ring(13),
                                   W.xxz_spin1_chain(9, seed=3)])
def test_tile_workload_shapes(capi, model):
    from plan_emulator import emulate_tile
    D = oracle.dimension(model.sites)
    x = W.vector(D, 4)
    T = capi.plan_export(model.sites, model.terms, 2 | (1 << 8))
    ref = oracle.apply(model.sites, model.terms, x).real
    assert np.linalg.norm(emulate_tile(T, x) - ref) <= 1e-13 * np.linalg.norm(ref)


def test_tile_split_of_the_benchmark_shapes(capi):
    T = capi.plan_export(*_m(W.ferrimagnet_chain(20)), 2 | (1 << 8))
    assert (T["F"], T["R"], T["nt"]) == (216, 36, 224) and T["nblk"] == 7776
    T = capi.plan_export(*_m(W.tavis_cummings(24, 64, seed=7)), 2 | (1 << 8))
    assert (T["F"], T["R"], T["nt"]) == (256, 64, 256)
    # boson last in the leaf: every high or mid spin's JC hop is a member of
    # one of two leaf-factor groups (sqrt(n_b) and sqrt(n_b + 1))
    assert T["G"] == 3


@pytest.mark.parametrize("dims,kinds", [((2,) * 12, None), ((2, 3) * 5, None), ((5, 4, 3, 6, 2, 2), None)])
@pytest.mark.parametrize("nvec", [1, 2])
def test_tile_tables_of_a_complex_h(capi, dims, kinds, nvec):
    """The tile kernel's tables of the real and imaginary parts (bit 3) of a
    complex H give H = H_re + i H_im on complex vectors."""
    from plan_emulator import emulate_tile
    m = W.random_model(list(dims), kinds, nterms=16, seed=6)
    n = len(dims)
    terms = m.terms + [(0, "Sy", -1, "I", 0.5), (1, "Sx", n - 1, "Sy", -0.3), (n - 1, "Sy", 2, "Sz", 0.2)]
    D = oracle.dimension(m.sites)
    xr, xi = W.vector(D, 11, nvec=nvec), W.vector(D, 12, nvec=nvec)
    parts = []
    for part in (0, 8):
        try:
            parts.append(capi.plan_export(m.sites, terms, part | 2 | (nvec << 8)))
        except capi.HmError as e:
            assert e.code == capi.HM_ERR_UNSUPPORTED
            pytest.skip("no tile form for this split")
    Tr, Ti = parts
    y = (emulate_tile(Tr, xr) - emulate_tile(Ti, xi)) + 1j * (emulate_tile(Tr, xi) + emulate_tile(Ti, xr))
    ref = oracle.apply(m.sites, terms, xr + 1j * xi, nvec=nvec)
    assert np.abs(ref.imag).max() > 0
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
