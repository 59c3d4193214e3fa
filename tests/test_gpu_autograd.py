"""The torch.autograd.Function over n solver steps (LBMSolve): its loss and gradients are
those of lbm_adjoint (checked against the FP64 oracle adjoint in test_gpu_adjoint.py), the
incoming gradient scales them, and a central difference of the loss in one inflow
coefficient agrees within 1 % (FP32 loss: relative noise ~1e-6 against a ~1e-3 change)."""
import numpy as np
import pytest
import torch

import scenes
from gpu_helpers import lib_solver, need_gpu

pytestmark = pytest.mark.gpu

DIMS = (24, 12, 10)
FACES = ("inlet", "outlet", "periodic", "periodic", "periodic", "periodic")
LOSS = dict(n=10, K=4, w_drag=1.0, w_ke=1.0, ke_x0=16, ke_x1=24)


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def setup():
    nx, ny, nz = DIMS
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.05, 0.0, 0.0))
    X, A = scenes.fibonacci_sphere((8.3, 6.1, 4.7), 2.2, 60)
    s = lib_solver(nx=nx, ny=ny, nz=nz, nu=0.03, faces=FACES, u_in=0.05, noise=0.01, seed=3)
    coef = torch.tensor(scenes.inflow_coefficients(0.004, seed=5), dtype=torch.float64)
    return s, rho, u, X, A, coef


def loss_of(s, rho, u, X, A, coef):
    from paper_2101_11856_gb300 import lbm_solve
    return lbm_solve(coef, torch.as_tensor(X, dtype=torch.float32), s, rho, u, area=A, **LOSS)


def test_gradients_equal_lbm_adjoint_and_scale():
    from paper_2101_11856_gb300 import lbm_solve
    s, rho, u, X, A, coef = setup()
    c = coef.clone().requires_grad_(True)
    Xt = torch.tensor(X, dtype=torch.float32, requires_grad=True)
    L = lbm_solve(c, Xt, s, rho, u, area=A, **LOSS)
    gc, gx = torch.autograd.grad(3.0 * L, (c, Xt))
    # the same run through the C ABI directly
    s.set_inflow(coef.numpy())
    s.set_solids(X.astype(np.float32), A)
    s.set_state(rho, u)
    L2, dc, dx = s.adjoint(LOSS["n"], LOSS["K"], LOSS["w_drag"], LOSS["w_ke"], LOSS["ke_x0"], LOSS["ke_x1"], 60)
    assert float(L.detach()) == L2                           # deterministic: bit-identical reruns
    assert np.allclose(gc.numpy(), 3.0 * dc, rtol=1e-12, atol=0)
    assert np.allclose(gx.numpy(), 3.0 * dx, rtol=1e-6, atol=1e-12)
    assert np.abs(dc).max() > 0 and np.abs(dx).max() > 0


def test_central_difference_in_one_coefficient():
    s, rho, u, X, A, coef = setup()
    c = coef.clone().requires_grad_(True)
    L = loss_of(s, rho, u, X, A, c)
    (g,) = torch.autograd.grad(L, (c,))
    k, h = 5, 2e-3
    e = torch.zeros(16, dtype=torch.float64)
    e[k] = h
    Lp = float(loss_of(s, rho, u, X, A, coef + e))
    Lm = float(loss_of(s, rho, u, X, A, coef - e))
    fd = (Lp - Lm) / (2 * h)
    print(f"dL/da_{k}: adjoint {float(g[k]):.6e}, central difference {fd:.6e}")
    assert abs(fd - float(g[k])) <= 1e-2 * abs(fd)
