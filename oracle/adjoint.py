"""Loss of the adjoint problem and its exact gradients (FP64 reverse mode).

ORACLE -- test infrastructure only.

The paper has no adjoint; the differentiable form of the solver asks for gradients of
a scalar loss of an n-step run with respect to the inflow-profile parameters and the
positions of the immersed-boundary samples.  The loss is

    L = w_drag * (1/n) sum_{t=1..n} D_x(t)  +  w_ke * 1/2 sum_{x0 <= x < x1} rho |u|^2 (t = n)

with D(t) = -sum_s g_s(t) the drag on the solid at step t (Algorithm 2, total force) and
rho, u the macroscopic fields of the last collision.  The inflow is
u_in(y, z) = u_in (1 + noise xi) + sum_mn a_mn sin(m pi (y+1/2)/ny) sin(n pi (z+1/2)/nz)
(16 coefficients a_mn).

The oracle's gradient is the definition itself: reverse-mode differentiation (PyTorch
autograd, a library primitive) of the FP64 forward steps in ``solver``; it is pinned
against central finite differences in ``tests/test_oracle_adjoint.py``.  Position
gradients exist where no sample crosses a cell face (the trilinear kernel is piecewise
linear in X; on a face the base cell's side is taken).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import collision as col
from .lattice import DTYPE
from .solver import Problem, step


@dataclass
class Loss:
    w_drag: float = 1.0
    w_ke: float = 1.0
    ke_x0: int = 0
    ke_x1: int = 0


def run_loss(p: Problem, rho, u, X, area, u_b, coef, n: int, loss: Loss):
    """Forward n steps from f = f_eq(rho, u) and return the scalar loss (differentiable)."""
    f = col.equilibrium(rho, u)
    drag_sum = torch.zeros((), dtype=DTYPE)
    diag = None
    for t in range(1, n + 1):
        f, diag = step(p, f, t, coef, (X, area, u_b))
        drag_sum = drag_sum + diag["drag"][0]
    ke = 0.5 * (diag["rho"] * (diag["u"] ** 2).sum(0))[:, :, loss.ke_x0:loss.ke_x1].sum()
    return loss.w_drag * drag_sum / n + loss.w_ke * ke


def loss_and_gradients(p: Problem, rho, u, X, area, u_b, coef, n: int, loss: Loss):
    """Return (L, dL/d coef (16,), dL/d X (S, 3)) for an n-step run."""
    rho = torch.as_tensor(np.asarray(rho), dtype=DTYPE)
    u = torch.as_tensor(np.asarray(u), dtype=DTYPE)
    Xt = torch.as_tensor(np.asarray(X), dtype=DTYPE).clone().requires_grad_(True)
    S = Xt.shape[0]
    area = torch.ones(S, dtype=DTYPE) if area is None else torch.as_tensor(np.asarray(area), dtype=DTYPE)
    u_b = torch.zeros(3, S, dtype=DTYPE) if u_b is None else torch.as_tensor(np.asarray(u_b), dtype=DTYPE).T
    ct = torch.as_tensor(np.asarray(coef), dtype=DTYPE).clone().requires_grad_(True)
    L = run_loss(p, rho, u, Xt, area, u_b, ct, n, loss)
    gc, gX = torch.autograd.grad(L, [ct, Xt], allow_unused=True)
    # a parameter the loss does not depend on (no inlet, no solid) has zero gradient
    gc = torch.zeros_like(ct) if gc is None else gc
    gX = torch.zeros_like(Xt) if gX is None else gX
    return float(L.detach()), gc.detach(), gX.detach()


def loss_value(p: Problem, rho, u, X, area, u_b, coef, n: int, loss: Loss) -> float:
    """Forward-only loss (for finite differences)."""
    with torch.no_grad():
        rho = torch.as_tensor(np.asarray(rho), dtype=DTYPE)
        u = torch.as_tensor(np.asarray(u), dtype=DTYPE)
        Xt = torch.as_tensor(np.asarray(X), dtype=DTYPE)
        S = Xt.shape[0]
        area = torch.ones(S, dtype=DTYPE) if area is None else torch.as_tensor(np.asarray(area), dtype=DTYPE)
        u_b = torch.zeros(3, S, dtype=DTYPE) if u_b is None else torch.as_tensor(np.asarray(u_b), dtype=DTYPE).T
        ct = torch.as_tensor(np.asarray(coef), dtype=DTYPE)
        return float(run_loss(p, rho, u, Xt, area, u_b, ct, n, loss))
