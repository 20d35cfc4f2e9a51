"""hm_coupling_gradients_static: coupling gradients for callers that cannot
let the library allocate device memory (stream capture, a foreign memory
pool). It keeps its partial sums in a fixed library-static device array and
must agree with hm_apply_adjoint, call after call.

This file is collected last, so a run that stops at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _entry():
    from paper_2606_02169_gb300 import _capi
    lib = _capi.load()
    f = lib.hm_coupling_gradients_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib, f


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_static_scratch_gradients_match_adjoint_twice(dtype):
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian
    lib, f = _entry()
    tdt = getattr(torch, dtype)
    code = 0 if dtype == "float64" else 1
    for m, nvec in ((W.square_lattice_xxz(3, 4, seed=4), 1), (W.ferrimagnet_chain(10), 3)):
        h = Hamiltonian(m.sites, m.terms)
        D = h.D
        gy = torch.from_numpy(W.vector(D, 5, nvec=nvec)).to("cuda", tdt)
        x = torch.from_numpy(W.vector(D, 6, nvec=nvec)).to("cuda", tdt)
        _, ref = h.adjoint(gy, x, want_gx=False)            # allocating entry point
        ref = ref.cpu().numpy()
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):                               # the array keeps the last call's data
            out = torch.full((h.nterms,), float("nan"), dtype=torch.float64, device="cuda")
            rc = f(h.handle, gy.data_ptr(), x.data_ptr(), out.data_ptr(), nvec, code, stream)
            assert rc == 0, lib.hm_last_error().decode()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            scale = np.abs(ref).max()
            assert np.allclose(got, ref, rtol=1e-11, atol=1e-13 * scale), (m.name, call)


def test_static_scratch_matches_oracle():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian
    lib, f = _entry()
    m = W.random_model([3, 2, 5, 2, 3, 4, 2, 3, 2], None, nterms=24, seed=1)
    D = oracle.dimension(m.sites)
    gy, x = W.vector(D, 1), W.vector(D, 2)
    h = Hamiltonian(m.sites, m.terms)
    out = torch.empty(h.nterms, dtype=torch.float64, device="cuda")
    gy_d, x_d = torch.from_numpy(gy).cuda(), torch.from_numpy(x).cuda()   # keep both alive
    rc = f(h.handle, gy_d.data_ptr(), x_d.data_ptr(), out.data_ptr(), 1, 0, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    ref = oracle.term_gradients(m.sites, m.terms, gy, x).real
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-11, atol=1e-12)


def test_static_scratch_rejects_term_lists_beyond_its_size():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian, _capi
    lib, f = _entry()
    terms = [(0, "Sz", -1, "I", 1e-6)] * 131073
    h = Hamiltonian([("spin", 2), ("spin", 2)], terms)
    v = torch.zeros(4, dtype=torch.float64, device="cuda")
    g = torch.zeros(131073, dtype=torch.float64, device="cuda")
    rc = f(h.handle, v.data_ptr(), v.data_ptr(), g.data_ptr(), 1, 0, None)
    assert rc == _capi.HM_ERR_TOO_LARGE
    assert "131072" in lib.hm_last_error().decode()


def test_static_scratch_checks_vectors_before_any_launch():
    """A misaligned gy, x or gcoef is refused on the host (the same checks as
    hm_apply_adjoint), so no kernel ever sees it."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian, _capi
    lib, f = _entry()
    m = W.square_lattice_xxz(2, 3, seed=4)
    h = Hamiltonian(m.sites, m.terms)
    buf = torch.zeros(h.D + 1, dtype=torch.float64, device="cuda")
    g = torch.zeros(h.nterms + 1, dtype=torch.float64, device="cuda")
    base, gbase = buf.data_ptr(), g.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    for gy, x, gc in ((base + 4, base, gbase), (base, base + 4, gbase), (base, base, gbase + 4)):
        rc = f(h.handle, gy, x, gc, 1, 0, stream)
        assert rc == _capi.HM_ERR_INVALID_ARG, lib.hm_last_error().decode()
    rc = f(h.handle, base, base, gbase, 1 << 20, 0, stream)        # nvec above 2^19
    assert rc == _capi.HM_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0                     # nothing was written


def test_static_scratch_allocates_no_device_memory():
    """After one warm call (kernel modules loaded, scratch address looked up),
    further calls leave the device's free memory and torch's allocator alone."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian
    lib, f = _entry()
    m = W.square_lattice_xxz(3, 4, seed=4)
    h = Hamiltonian(m.sites, m.terms)
    gy = torch.from_numpy(W.vector(h.D, 5)).cuda()
    x = torch.from_numpy(W.vector(h.D, 6)).cuda()
    out = torch.empty(h.nterms, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert f(h.handle, gy.data_ptr(), x.data_ptr(), out.data_ptr(), 1, 0, stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert f(h.handle, gy.data_ptr(), x.data_ptr(), out.data_ptr(), 1, 0, stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_static_scratch_gradients_in_a_cuda_graph(dtype):
    """Captured into a CUDA graph (after one warm call) and replayed on new
    gy and x copied into the captured buffers: each replay equals an
    uncaptured call on those vectors bit for bit, and hm_apply_adjoint's
    gradients within the FP64 tolerance (their grids differ)."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Hamiltonian
    lib, f = _entry()
    tdt = getattr(torch, dtype)
    code = 0 if dtype == "float64" else 1
    m = W.square_lattice_xxz(3, 4, seed=4)
    h = Hamiltonian(m.sites, m.terms)
    gy = torch.from_numpy(W.vector(h.D, 7)).to("cuda", tdt)
    x = torch.from_numpy(W.vector(h.D, 8)).to("cuda", tdt)
    out = torch.empty(h.nterms, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):                       # warm call outside the capture
        assert f(h.handle, gy.data_ptr(), x.data_ptr(), out.data_ptr(), 1, code, side.cuda_stream) == 0
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rc = f(h.handle, gy.data_ptr(), x.data_ptr(), out.data_ptr(), 1, code, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    for seed in (11, 12):
        gy.copy_(torch.from_numpy(W.vector(h.D, seed)).to(tdt))
        x.copy_(torch.from_numpy(W.vector(h.D, seed + 50)).to(tdt))
        g.replay()
        torch.cuda.synchronize()
        got = out.clone()
        direct = torch.full_like(out, float("nan"))
        rc = f(h.handle, gy.data_ptr(), x.data_ptr(), direct.data_ptr(), 1, code,
               torch.cuda.current_stream().cuda_stream)
        assert rc == 0
        _, ref = h.adjoint(gy, x, want_gx=False)
        torch.cuda.synchronize()
        assert torch.equal(got, direct), seed
        r = ref.cpu().numpy()
        assert np.allclose(got.cpu().numpy(), r, rtol=1e-11, atol=1e-13 * np.abs(r).max()), seed
