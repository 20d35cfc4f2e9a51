"""torch.autograd wrappers over the hm kernels.

HamApply:  y = H(c) x. Backward runs the hand-written adjoint kernel:
           dL/dx = H^T gy and dL/dc_t = <gy| O_t |x> for every term t.
LanczosE0: E0(c) from the device Lanczos driver. Backward uses
           Hellmann-Feynman, dE0/dc_t = <psi0| O_t |psi0>, with psi0 rebuilt
           by recomputation (no stored Krylov basis).
Physical couplings (J, Delta, h, ...) map to the term coefficients c with
ordinary differentiable torch ops; the chain rule to them is torch's.
"""
from __future__ import annotations

import torch

from .hamiltonian import Hamiltonian


def _sync_coefs(ham: Hamiltonian, coefs: torch.Tensor):
    """Bring the plan's coefficients up to date with `coefs`. The plan's
    tables are rebuilt on the host, so a changed coefficient tensor costs one
    device-to-host read; an unchanged one (the same tensor, not modified in
    place since the last call: same version counter) costs nothing and does
    not synchronise the host."""
    ref = getattr(ham, "_coef_ref", None)
    if ref is not None and ref[0] is coefs and ref[1] == coefs._version:
        return
    c = coefs.detach().double().cpu().tolist()
    if c != ham.coefs:
        ham.set_coefficients(c)
    ham._coef_ref = (coefs, coefs._version)   # holds the tensor: its identity stays unique


class HamApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coefs: torch.Tensor, x: torch.Tensor, ham: Hamiltonian):
        _sync_coefs(ham, coefs)
        y = ham.apply(x.contiguous())
        ctx.save_for_backward(x)
        ctx.ham = ham
        ctx.cdev, ctx.cdt = coefs.device, coefs.dtype
        return y

    @staticmethod
    def backward(ctx, gy):
        (x,) = ctx.saved_tensors
        want_gc, want_gx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gx, gc = ctx.ham.adjoint(gy.contiguous().to(x.dtype), x, want_gx=want_gx, want_gcoef=want_gc)
        if gc is not None:
            gc = gc.to(device=ctx.cdev, dtype=ctx.cdt)
        return gc, gx, None


def hamiltonian_apply(ham: Hamiltonian, coefs: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    return HamApply.apply(coefs, x, ham)


class LanczosE0(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coefs: torch.Tensor, v0: torch.Tensor, ham: Hamiltonian, steps: int, reorth: bool):
        _sync_coefs(ham, coefs)
        r = ham.lanczos(v0.contiguous(), steps, reorth=reorth, ritz_vector=True)
        ctx.save_for_backward(r["psi0"])
        ctx.ham = ham
        ctx.cdev, ctx.cdt = coefs.device, coefs.dtype
        return torch.tensor(r["e0"], dtype=torch.float64, device=coefs.device)

    @staticmethod
    def backward(ctx, ge):
        (psi,) = ctx.saved_tensors
        _, gc = ctx.ham.adjoint(psi, psi, want_gx=False, want_gcoef=True)
        return (gc * ge.to(gc.device)).to(device=ctx.cdev, dtype=ctx.cdt), None, None, None, None


def lanczos_e0(ham: Hamiltonian, coefs: torch.Tensor, v0: torch.Tensor, steps: int = 100,
               reorth: bool = True) -> torch.Tensor:
    return LanczosE0.apply(coefs, v0, ham, steps, reorth)
