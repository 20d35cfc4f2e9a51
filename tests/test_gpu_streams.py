"""Applies of one plan from several streams, and FP64 applies recorded in a
CUDA graph: the FP64 input split takes per-call stream-ordered scratch, so
neither case shares a buffer between calls that may overlap."""
import pytest

import workloads as W
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _ham(m):
    from paper_2606_02169_gb300 import Hamiltonian
    return Hamiltonian(m.sites, m.terms)


def test_fp64_applies_of_one_plan_on_two_streams():
    torch = torch_cuda()
    h = _ham(W.xxz_spin1_chain(13, seed=71))          # D = 3^13
    xa = torch.from_numpy(W.vector(h.D, 1)).cuda()
    xb = torch.from_numpy(W.vector(h.D, 2)).cuda()
    want_a, want_b = h.apply(xa), h.apply(xb)
    ya, yb = torch.empty_like(xa), torch.empty_like(xb)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(8):
        h.apply(xa, out=ya, stream=sa)
        h.apply(xb, out=yb, stream=sb)
    torch.cuda.synchronize()
    assert torch.equal(ya, want_a)
    assert torch.equal(yb, want_b)


def test_fp64_apply_recorded_in_a_graph_at_a_new_size():
    """Warm-up at nvec=1, capture at nvec=2: the capture needs no scratch of
    that size beforehand."""
    torch = torch_cuda()
    h = _ham(W.xxz_spin1_chain(9, seed=72))
    h.apply(torch.from_numpy(W.vector(h.D, 3)).cuda())
    x = torch.from_numpy(W.vector(h.D, 4, nvec=2)).cuda()
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        h.apply(x, out=y, stream=s)
    want = h.apply(x)
    for _ in range(2):
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y, want)


def test_fp64_batch_recorded_in_a_graph():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch
    hams = [_ham(m) for m in W.disorder_ensemble(count=5, nmin=3, nmax=6, base_seed=73)]
    xs = [torch.from_numpy(W.vector(h.D, 10 + i, nvec=3)).cuda() for i, h in enumerate(hams)]
    ys = [torch.empty_like(x) for x in xs]
    b = Batch(hams)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.apply(xs, ys, stream=s)   # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.apply(xs, ys, stream=s)
    for y in ys:
        y.zero_()
    g.replay()
    torch.cuda.synchronize()
    for h, x, y in zip(hams, xs, ys):
        assert torch.equal(h.apply_ex(x, kernel="general"), y)   # batches run the general kernel
