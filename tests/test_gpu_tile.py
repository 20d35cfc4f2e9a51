"""The leaf-tiled apply kernel (hm_apply_ex with the tile bit) against the
oracle, element by element: FP64 (double-float and native), FP32, several
right-hand sides, H^T, and the shapes without a tile form."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ((3, 2, 4, 2, 3), None),                                   # one block, no high sites
    ((3, 2, 5, 2, 3, 4, 2, 3, 2), None),
    ((2,) * 14, None),
    ((2,) * 16, None),                                         # several blocks, high sites
    ((2, 3) * 6, None),
    ((3,) * 10, None),
    ((64, 2, 2, 2, 2, 2, 2, 2), ["boson"] + ["spin"] * 7),
    ((2, 2, 2, 2, 2, 2, 2, 64), ["spin"] * 7 + ["boson"]),
    ((3, 5, 2, 7, 3, 2, 2, 3), ["spin", "boson", "spin", "boson", "spin", "spin", "spin", "spin"]),
]


def _run(torch, h, x, dtype, **kw):
    xd = torch.from_numpy(x).to("cuda", torch.float64 if dtype == np.float64 else torch.float32)
    y = h.apply_ex(xd, kernel="tile", **kw)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("dims,kinds", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tile_matches_oracle(dims, kinds, dtype):
    torch = torch_cuda()
    m = W.random_model(list(dims), kinds, nterms=28, seed=21)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 22)
    if dtype == np.float32:
        x = x.astype(np.float32).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x)
    got = _run(torch, ham(m), x, dtype)
    check_close(got, ref, abs_bound(m, x), TOL_F64 if dtype == np.float64 else TOL_F32, f"tile {dims}")


@pytest.mark.parametrize("dims,kinds", CASES[2:6])
def test_tile_native_fp64(dims, kinds):
    torch = torch_cuda()
    m = W.random_model(list(dims), kinds, nterms=28, seed=23)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 24)
    ref = oracle.apply(m.sites, m.terms, x)
    got = _run(torch, ham(m), x, np.float64, native_f64=True)
    check_close(got, ref, abs_bound(m, x), 1e-13, f"tile native {dims}")


@pytest.mark.parametrize("nvec", [2, 3, 16])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tile_multiple_right_hand_sides(nvec, dtype):
    torch = torch_cuda()
    m = W.random_model([3, 2, 4, 2, 3, 2, 5, 2], None, nterms=30, seed=25)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 26, nvec=nvec).astype(dtype).astype(np.float64)
    ref = oracle.apply(m.sites, m.terms, x, nvec=nvec)
    got = _run(torch, ham(m), x, dtype)
    check_close(got, ref, abs_bound(m, x), TOL_F64 if dtype == np.float64 else TOL_F32, f"tile nvec={nvec}")


@pytest.mark.parametrize("dims,kinds", [CASES[1], CASES[3], CASES[8]])
def test_tile_transpose(dims, kinds):
    torch = torch_cuda()
    m = W.random_model(list(dims), kinds, nterms=28, seed=27, hermitian=False)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 28)
    H = oracle.dense(m.sites, m.terms, sparse=True)
    ref = np.asarray(H.T @ x).real
    got = _run(torch, ham(m), x, np.float64, transpose=True)
    scale = np.asarray(abs(H).T @ np.abs(x)).reshape(-1)
    check_close(got, ref, scale, TOL_F64, f"tile H^T {dims}")


def test_tile_workloads_agree_with_general_kernel():
    torch = torch_cuda()
    for m in (W.ferrimagnet_chain(14), W.tavis_cummings(10, 16, seed=2), W.square_lattice_xxz(3, 5, seed=4)):
        h = ham(m)
        D = oracle.dimension(m.sites)
        x = W.vector(D, 3)
        ref = oracle.apply(m.sites, m.terms, x)
        scale = abs_bound(m, x)
        for dtype in (np.float64, np.float32):
            xv = x if dtype == np.float64 else x.astype(np.float32).astype(np.float64)
            refv = ref if dtype == np.float64 else oracle.apply(m.sites, m.terms, xv)
            check_close(_run(torch, h, xv, dtype), refv, scale, TOL_F64 if dtype == np.float64 else TOL_F32,
                        "tile workload")


def test_no_tile_form_is_reported():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError
    m = W.random_model([4500], ["boson"], nterms=6, seed=1)
    h = ham(m)
    x = torch.zeros(h.D, dtype=torch.float64, device="cuda")
    with pytest.raises(HmError):
        h.apply_ex(x, kernel="tile")
    y = h.apply(x)   # the library's kernel
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0
