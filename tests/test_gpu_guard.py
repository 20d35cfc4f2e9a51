"""Guard bands (a stand-in for a memory checker): every vector a kernel reads
or writes sits inside a larger buffer whose elements before and after it are
NaN. After each call the guards must be untouched, bit for bit (no write out
of bounds), and the results must equal the oracle's, finite (a read of a
guard element, even one multiplied by a zero coefficient, would turn a
result into NaN). Ragged shapes, odd guard offsets (vectors starting off a
16-byte boundary), every apply kernel and launch variant, the adjoint, the
batch, a sector plan, complex vectors, Lanczos and time evolution."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import TOL_F32, TOL_F64, abs_bound, check_close, ham, torch_cuda

pytestmark = pytest.mark.gpu


class Guarded:
    """A vector of n elements at offset g inside a NaN buffer of n + 2g."""

    def __init__(self, torch, n, dtype, g, values=None):
        self.torch, self.n, self.g = torch, n, g
        nan = complex(float("nan"), float("nan")) if dtype.is_complex else float("nan")
        self.buf = torch.full((n + 2 * g,), nan, dtype=dtype, device="cuda")
        self.v = self.buf[g:g + n]
        if values is not None:
            self.v.copy_(torch.as_tensor(values).to(self.buf.dtype).cuda())

    def guards_intact(self):
        b = self.buf.cpu()
        head, tail = b[:self.g], b[self.g + self.n:]
        if self.buf.is_complex():
            return bool(head.real.isnan().all() and head.imag.isnan().all() and tail.real.isnan().all()
                        and tail.imag.isnan().all())
        return bool(head.isnan().all() and tail.isnan().all())


SHAPES = [
    ((3, 2, 5, 2, 3, 4, 2, 3, 2), None),
    ((2, 2, 2, 2, 2, 2, 2, 64), ["spin"] * 7 + ["boson"]),
    ((2, 3) * 5, None),
]
VARIANTS = [dict(), dict(kernel="general", small=True), dict(kernel="general", prefetch=True, s=4),
            dict(kernel="staged"), dict(kernel="tile")]


@pytest.mark.parametrize("dims,kinds", SHAPES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("nvec,g", [(1, 1), (3, 3), (1, 16)])
def test_apply_stays_inside_its_vectors(dims, kinds, dtype, nvec, g):
    torch = torch_cuda()
    from paper_2606_02169_gb300 import HmError
    m = W.random_model(list(dims), kinds, nterms=26, seed=30, hermitian=False)
    D = oracle.dimension(m.sites)
    x = W.vector(D, 31, nvec=nvec).astype(dtype).astype(np.float64)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    tol = TOL_F64 if dtype == np.float64 else TOL_F32
    ref = oracle.apply(m.sites, m.terms, x, nvec=nvec)
    h = ham(m)
    gx = Guarded(torch, D * nvec, tdt, g, x)
    for kw in VARIANTS:
        for transpose in (False, True):
            gy = Guarded(torch, D * nvec, tdt, g)
            try:
                if kw:
                    h.apply_ex(gx.v, out=gy.v, transpose=transpose, **kw)
                elif transpose:
                    h.apply_ex(gx.v, out=gy.v, transpose=True)
                else:
                    h.apply(gx.v, out=gy.v)
            except HmError:
                assert kw.get("kernel") == "tile"   # no tile form for this shape or nvec
                continue
            torch.cuda.synchronize()
            assert gy.guards_intact(), f"write outside y: {kw} transpose={transpose}"
            assert gx.guards_intact()
            got = gy.v.double().cpu().numpy()
            assert np.isfinite(got).all(), f"a guard element was read: {kw} transpose={transpose}"
            if not transpose:
                check_close(got, ref, abs_bound(m, x), tol, f"{kw}")
    from paper_2606_02169_gb300 import _capi
    assert _capi.device_status() == 0


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_adjoint_batch_sector_complex_stay_inside(dtype):
    torch = torch_cuda()
    from paper_2606_02169_gb300 import Batch, Hamiltonian
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    g = 5
    # adjoint: gx and the coupling gradients
    m = W.random_model([3, 2, 4, 2, 3], None, nterms=20, seed=40)
    h = ham(m)
    D = h.D
    gy = Guarded(torch, D, tdt, g, W.vector(D, 41))
    xx = Guarded(torch, D, tdt, g, W.vector(D, 42))
    gxv = Guarded(torch, D, tdt, g)
    gcv = Guarded(torch, h.nterms, torch.float64, g)
    h.adjoint(gy.v, xx.v, gx=gxv.v, gcoef=gcv.v)
    torch.cuda.synchronize()
    for gv in (gy, xx, gxv, gcv):
        assert gv.guards_intact()
    assert torch.isfinite(gxv.v).all() and torch.isfinite(gcv.v).all()
    # batch of uneven instances
    models = W.disorder_ensemble(count=5, nmin=3, nmax=6, base_seed=43)
    hams = [ham(mm) for mm in models]
    xs = [Guarded(torch, hh.D * 2, tdt, g, W.vector(hh.D, 44 + i, nvec=2)) for i, hh in enumerate(hams)]
    ys = [Guarded(torch, hh.D * 2, tdt, g) for hh in hams]
    Batch(hams).apply([v.v for v in xs], [v.v for v in ys])
    torch.cuda.synchronize()
    for v in xs + ys:
        assert v.guards_intact()
    assert all(bool(torch.isfinite(v.v).all()) for v in ys)
    # sector plan
    n = 12
    sites = [("spin", 2)] * n
    terms = []
    for i in range(n):
        j = (i + 1) % n
        terms += [(i, "Sp", j, "Sm", 0.5), (i, "Sm", j, "Sp", 0.5), (i, "Sz", j, "Sz", 1.0)]
    hs = Hamiltonian(sites, terms, sector_total=n // 2)
    sx = Guarded(torch, hs.D, tdt, g, W.vector(hs.D, 45))
    sy = Guarded(torch, hs.D, tdt, g)
    hs.apply(sx.v, out=sy.v)
    torch.cuda.synchronize()
    assert sx.guards_intact() and sy.guards_intact() and bool(torch.isfinite(sy.v).all())
    # complex vector of a real H, and Lanczos / time evolution outputs
    cdt = torch.complex128 if dtype == np.float64 else torch.complex64
    hc = ham(W.ferrimagnet_chain(6))
    cx = Guarded(torch, hc.D, cdt, g, W.vector(hc.D, 46) + 1j * W.vector(hc.D, 47))
    cy = Guarded(torch, hc.D, cdt, g)
    hc.apply(cx.v, out=cy.v)
    torch.cuda.synchronize()
    assert cx.guards_intact() and cy.guards_intact()
    v0 = Guarded(torch, hc.D, tdt, g, W.vector(hc.D, 48))
    r = hc.lanczos(v0.v, 40, reorth=True, ritz_vector=True)
    torch.cuda.synchronize()
    assert v0.guards_intact() and np.isfinite(r["e0"]) and bool(torch.isfinite(r["psi0"]).all())
    if dtype == np.float64:
        ev = Guarded(torch, hc.D, torch.complex128, g)
        hc.evolve(cx.v, 0.3, m=20, out=ev.v)
        torch.cuda.synchronize()
        assert ev.guards_intact() and cx.guards_intact()
