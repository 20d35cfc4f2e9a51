"""Launch variants the autotuner chooses between (kernel, elements per thread
S, register cap, grid size): each one matches the oracle, and all launches of
one kernel give the same y bit for bit, so tuning never changes a result
beyond the choice of kernel."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [2, 3, 4, 6, 8]
TILE_ROWS = [1, 2, 4]

MODELS = [
    ((3, 2, 5, 2, 3, 4, 2, 3, 2), None),                 # ragged low block, 1 high site
    ((2,) * 14, None),                                     # 2 high sites
    ((3, 5, 2, 7, 3, 2, 2, 3), ["spin", "boson", "spin", "boson", "spin", "spin", "spin", "spin"]),
]


def _to(torch, a, dtype):
    return torch.from_numpy(a).to("cuda", torch.float64 if dtype == np.float64 else torch.float32)


@pytest.mark.parametrize("dims,kinds", MODELS)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("nvec", [1, 3])
def test_every_variant_matches_oracle_and_each_other(dims, kinds, dtype, nvec):
    torch = torch_cuda()
    m = W.random_model(list(dims), kinds, nterms=28, seed=11)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 12, nvec=nvec)
    if dtype == np.float32:
        x = x.astype(np.float32).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x, nvec=nvec)
    scale = abs_bound(m, x)
    tol = TOL_F64 if dtype == np.float64 else TOL_F32
    h = ham(m)
    xd = _to(torch, x, dtype)
    for kernel, small, shapes, mbs in (("general", False, SHAPES, (False, True)),
                                       ("general", True, SHAPES, (False, True)),
                                       ("tile", False, TILE_ROWS, (False,)),
                                       ("staged", False, [0], (False,))):
        base = h.apply_ex(xd, kernel=kernel, small=small)
        torch.cuda.synchronize()
        check_close(base.double().cpu().numpy(), ref, scale, tol, f"{kernel} small={small} default launch")
        for s in shapes:
            for mb in mbs:
                for ctas in (0, 7):
                    y = h.apply_ex(xd, s=s, mb=mb, ctas=ctas, kernel=kernel, small=small)
                    torch.cuda.synchronize()
                    assert torch.equal(y, base), \
                        f"{kernel} small={small} S={s} mb={mb} ctas={ctas} differs from its default"
        if kernel == "general":
            # the prefetching variant sums in the same order: bit for bit
            for s in (4, 6, 8):
                for mb in mbs:
                    y = h.apply_ex(xd, s=s, mb=mb, kernel=kernel, small=small, prefetch=True)
                    torch.cuda.synchronize()
                    assert torch.equal(y, base), f"prefetch small={small} S={s} mb={mb} differs"


def test_invalid_elements_per_thread_is_rejected():
    torch = torch_cuda()
    m = W.heisenberg_ring(6)
    h = ham(m)
    x = torch.zeros(h.D, dtype=torch.float64, device="cuda")
    for bad in (1, 5, 7, 9, 15):
        with pytest.raises(RuntimeError):
            h.apply_ex(x, s=bad)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tuned_apply_matches_its_kernel(dtype):
    torch = torch_cuda()
    m = W.ferrimagnet_chain(10)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 4)
    h = ham(m)
    xd = _to(torch, x, dtype)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    cfg = h.tune(1, tdt)
    assert cfg == h.tuned_config(1, tdt)
    assert cfg["kernel"] in (1, 2, 3) and cfg["ctas"] >= 0 and cfg["mb"] in (0, 1)
    assert cfg["s"] in {1: [0] + SHAPES, 2: [0] + TILE_ROWS, 3: [0]}[cfg["kernel"]]
    y1 = h.apply(xd)
    kernel = {1: "general", 2: "tile", 3: "staged"}[cfg["kernel"]]
    y2 = h.apply_ex(xd, kernel=kernel, s=cfg["s"], mb=bool(cfg["mb"]), ctas=cfg["ctas"], small=bool(cfg["small"]),
                    prefetch=bool(cfg["prefetch"]), scalar=bool(cfg["scalar"]), split=bool(cfg["split"]),
                    split_sites=cfg["split_sites"], vinv=bool(cfg["vinv"]))
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    # a second plan with the same signature takes the cached choice without timing
    h2 = ham(m)
    assert h2.tuned_config(1, tdt) == cfg
    gx, _ = h.adjoint(xd, want_gcoef=False)
    torch.cuda.synchronize()
    ref = oracle.apply(m.sites, m.terms, x)
    check_close(y1.double().cpu().numpy(), ref, abs_bound(m, x), TOL_F64 if dtype == np.float64 else TOL_F32,
                "tuned")
    # ferrimagnet chain: real symmetric, so H^T gy = H gy with the same tables
    assert torch.equal(gx, y1)
