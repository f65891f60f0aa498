"""torch.autograd front end of dirac_adjoint_gradient.

``propagated_observable(V_blocks, coef, setup)`` is a differentiable scalar:
the observable of the final state after ``setup.nsteps`` steps of the FP64
propagator with the potential energy V constant on blocks of
``setup.block`` = (by, bx) sites (V_blocks has shape (ny / by, nx / bx)) and
the step-mean vector potential A_x of step n equal to (W coef)_n (W: the step
means of the pulse basis, e.g. a sine series).  The gradient with respect to
both inputs comes from the library's adjoint sweep (one call computes the
observable and, when an input requires grad, its gradients).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .propagator import Propagator


@dataclasses.dataclass
class AdjointSetup:
    nx: int
    ny: int
    dx: float
    dy: float
    psi0: object              # CUDA complex128 (ny, nx, 2)
    dt: float
    m: int
    nsteps: int
    W: np.ndarray             # (nsteps, n_coef)
    observable: str = "px"    # "px" or "proj"
    phi: object = None        # CUDA complex128 (ny, nx, 2) for "proj"
    block: tuple = (1, 1)     # (by, bx)
    checkpoint_every: int = 50
    shift: float = 0.0
    order: int = 2
    boundary: str = "periodic"
    mass: float = 1.0
    c: float = 137.036
    _prop: Propagator = None

    def propagator(self) -> Propagator:
        if self._prop is None:
            self._prop = Propagator(self.nx, self.ny, self.dx, self.dy, mass=self.mass, c=self.c,
                                    order=self.order, boundary=self.boundary, m_max=self.m)
        return self._prop


def _torch():
    import torch
    return torch


class PropagatedObservable(_torch().autograd.Function):
    @staticmethod
    def forward(ctx, V_blocks, coef, setup: AdjointSetup):
        torch = _torch()
        by, bx = setup.block
        V = V_blocks.detach().to(torch.float64).repeat_interleave(by, 0).repeat_interleave(bx, 1)
        prop = setup.propagator()
        prop.set_fields(V.contiguous(), shift=setup.shift)
        A = np.zeros((setup.nsteps, 2))
        A[:, 0] = setup.W @ coef.detach().cpu().numpy().astype(np.float64)
        need_v, need_a = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        res = prop.adjoint_gradient(setup.psi0, setup.nsteps, setup.dt, setup.m, A,
                                    observable=setup.observable, phi=setup.phi,
                                    checkpoint_every=setup.checkpoint_every, block=setup.block,
                                    W=setup.W, grad_V=need_v, grad_A=need_a)
        dV = res.dV if need_v else torch.zeros_like(V_blocks, dtype=torch.float64)
        da = torch.from_numpy(res.da).to(coef.device) if need_a else torch.zeros_like(coef)
        ctx.save_for_backward(dV, da)
        return torch.tensor(res.loss, dtype=torch.float64, device=V_blocks.device)

    @staticmethod
    def backward(ctx, grad_out):
        dV, da = ctx.saved_tensors
        return grad_out * dV, grad_out * da, None


def propagated_observable(V_blocks, coef, setup: AdjointSetup):
    """Differentiable observable of the propagated state (see the module docstring)."""
    return PropagatedObservable.apply(V_blocks, coef, setup)
