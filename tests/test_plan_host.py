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
