"""Batched persistent apply over uneven instances vs per-instance applies of
the general kernel (bit-identical: the same block code for queued and
plainly launched members) and vs the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu


def test_batch_equals_single_applies_and_oracle():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch
    models = W.disorder_ensemble(count=12, nmin=3, nmax=8, base_seed=50)
    hams = [ham(m) for m in models]
    nvec = 16
    xs = [torch.from_numpy(W.vector(h.D, 100 + i, nvec=nvec)).to("cuda", torch.float32)
          for i, h in enumerate(hams)]
    b = Batch(hams)
    ys = b.apply(xs)
    torch.cuda.synchronize()
    for i, (m, h) in enumerate(zip(models, hams)):
        single = h.apply_ex(xs[i], kernel="general")
        assert torch.equal(single, ys[i]), i
        if h.D <= 3 ** 7:
            xn = xs[i].double().cpu().numpy()
            ref = oracle.apply(m.sites, m.terms, xn, nvec=nvec)
            check_close(ys[i].double().cpu().numpy(), ref, abs_bound(m, xn), TOL_F32, m.name)


def test_batch_graph_capture():
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch
    models = W.disorder_ensemble(count=6, nmin=3, nmax=6, base_seed=7)
    hams = [ham(m) for m in models]
    xs = [torch.from_numpy(W.vector(h.D, i, nvec=4)).to("cuda", torch.float32) for i, h in enumerate(hams)]
    ys = [torch.empty_like(x) for x in xs]
    b = Batch(hams)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.apply(xs, ys)            # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.apply(xs, ys, stream=s)
    for y in ys:
        y.zero_()
    g.replay()
    torch.cuda.synchronize()
    for h, x, y in zip(hams, xs, ys):
        assert torch.equal(h.apply_ex(x, kernel="general"), y)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_mixing_large_and_small_instances(dtype):
    """Instances that fill the GPU alone take plain launches, the rest the
    persistent work queue; results equal per-instance applies of the general
    kernel either way."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch
    from gpu_util import TOL_F64, apply_abs_bound
    models = [W.xxz_spin1_chain(13, seed=61)] + W.disorder_ensemble(count=5, nmin=3, nmax=7, base_seed=62) + \
        [W.xxz_spin1_chain(12, seed=63)]
    hams = [ham(m) for m in models]
    nvec = 2
    tdt = torch.float32 if dtype == "f32" else torch.float64
    xs = [torch.from_numpy(W.vector(h.D, 200 + i, nvec=nvec)).to("cuda", tdt) for i, h in enumerate(hams)]
    ys = Batch(hams).apply(xs)
    torch.cuda.synchronize()
    for i, h in enumerate(hams):
        assert torch.equal(h.apply_ex(xs[i], kernel="general"), ys[i]), i
    # the large instance against the oracle, every row
    xn = xs[0].double().cpu().numpy()
    ref = oracle.apply(models[0].sites, models[0].terms, xn, nvec=nvec)
    scale = apply_abs_bound(models[0], xn, nvec=nvec)
    check_close(ys[0].double().cpu().numpy(), ref, scale, TOL_F32 if dtype == "f32" else TOL_F64, "large")


def test_tuned_large_member_takes_its_tuned_launch():
    """A member that fills the GPU alone runs the launch hm_apply makes for
    it; after hm_tune that is the tuned choice (here possibly a split or
    vector-lane variant), and the queued members still equal the general
    kernel bit for bit."""
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch
    models = [W.xxz_spin1_chain(13, seed=81)] + W.disorder_ensemble(count=4, nmin=3, nmax=6, base_seed=82)
    hams = [ham(m) for m in models]
    nvec = 16
    hams[0].tune(nvec, torch.float32)
    xs = [torch.from_numpy(W.vector(h.D, 400 + i, nvec=nvec)).to("cuda", torch.float32) for i, h in enumerate(hams)]
    ys = Batch(hams).apply(xs)
    torch.cuda.synchronize()
    assert torch.equal(hams[0].apply(xs[0]), ys[0])
    for i in range(1, len(hams)):
        assert torch.equal(hams[i].apply_ex(xs[i], kernel="general"), ys[i]), i
