"""hm_apply on vectors in pinned host memory: the kernels read x and write y
over the CPU-GPU link (FP64: the split pass reads x once; FP32: x is first
copied once into device scratch). Results equal the same call on device
vectors bit for bit, on one stream and with calls alternating between two
streams; pageable host memory is rejected."""
import numpy as np
import pytest

import workloads as W
from gpu_util import ham, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,nvec", [("f64", 1), ("f32", 1), ("f64", 2), ("f32", 4), ("c128", 1)])
def test_pinned_host_vectors_match_device_vectors(dtype, nvec):
    torch = torch_cuda()
    m = W.random_model([2, 3, 2, 3, 2, 3, 2, 3, 2, 3, 2], None, nterms=30, seed=4)
    h = ham(m)
    tdt = {"f64": torch.float64, "f32": torch.float32, "c128": torch.complex128}[dtype]
    xn = W.vector(h.D, 8, nvec=nvec)
    if dtype == "c128":
        xn = xn + 1j * W.vector(h.D, 9, nvec=nvec)
    xd = torch.from_numpy(xn).to("cuda", tdt)
    yd = h.apply(xd)
    for host_x, host_y in ((True, False), (False, True), (True, True)):
        x = xd.cpu().pin_memory() if host_x else xd
        y = torch.empty(xd.shape, dtype=tdt, pin_memory=True) if host_y else torch.empty_like(xd)
        h.apply(x, out=y)
        torch.cuda.synchronize()
        assert torch.equal(y.cpu(), yd.cpu()), (host_x, host_y)
    # the binding allocates a pinned output for a pinned input
    yp = h.apply(xd.cpu().pin_memory())
    torch.cuda.synchronize()
    assert yp.is_pinned() and torch.equal(yp, yd.cpu())


def test_pageable_host_vectors_are_rejected():
    torch = torch_cuda()
    import ctypes
    from paper_2606_02169_gb300 import _capi as C
    m = W.random_model([2, 3, 2, 3, 2, 3], None, nterms=10, seed=1)
    h = ham(m)
    xd = torch.from_numpy(W.vector(h.D, 1)).cuda()
    yd = torch.empty_like(xd)
    xp = np.zeros(h.D)          # plain pageable host memory
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = h._lib.hm_apply(h._h, xp.ctypes.data, yd.data_ptr(), 1, C.HM_F64, s)
    assert rc == C.HM_ERR_INVALID_ARG
    rc = h._lib.hm_apply(h._h, xd.data_ptr(), xp.ctypes.data, 1, C.HM_F64, s)
    assert rc == C.HM_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        h.apply(torch.from_numpy(xp))


def test_host_vector_calls_on_two_streams():
    torch = torch_cuda()
    m = W.random_model([2, 3, 2, 3, 2, 3, 2, 3, 2, 3], None, nterms=30, seed=6)
    h = ham(m)
    xs = [torch.from_numpy(W.vector(h.D, 20 + i)) .pin_memory() for i in range(4)]
    ys = [torch.empty(h.D, dtype=torch.float64, pin_memory=True) for _ in range(4)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for i in range(4):
        h.apply(xs[i], out=ys[i], stream=streams[i % 2])
    torch.cuda.synchronize()
    for i in range(4):
        assert torch.equal(ys[i], h.apply(xs[i].cuda()).cpu()), i
