"""Pin of the oracle's adjoint gradients against central finite differences (no GPU)."""
import numpy as np
import pytest
import torch

import scenes
from oracle.adjoint import Loss, loss_and_gradients, loss_value
from oracle.solver import Problem


def small_channel():
    nx, ny, nz = 14, 8, 8
    p = Problem(nx, ny, nz, nu=0.05, u_in=0.04, noise=0.01, seed=7,
                faces=("inlet", "outlet", "periodic", "periodic", "periodic", "periodic"))
    X, A = scenes.fibonacci_sphere((5.3, 3.6, 3.4), 1.7, 24)
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0, 0))
    coef = np.random.default_rng(1).uniform(-0.005, 0.005, 16)
    return p, rho, u, X, A, coef


@pytest.mark.parametrize("loss", [Loss(1.0, 0.0), Loss(0.0, 1.0, 9, 14), Loss(1.0, 2.0, 10, 13)])
def test_gradients_match_central_differences(loss):
    p, rho, u, X, A, coef = small_channel()
    n = 6
    L, gc, gX = loss_and_gradients(p, rho, u, X, A, None, coef, n, loss)
    h = 1e-6
    for k in (0, 5, 15):
        cp, cm = coef.copy(), coef.copy()
        cp[k] += h
        cm[k] -= h
        fd = (loss_value(p, rho, u, X, A, None, cp, n, loss) - loss_value(p, rho, u, X, A, None, cm, n, loss)) / (2 * h)
        assert abs(fd - float(gc[k])) <= 1e-6 * max(abs(fd), 1e-3 * float(gc.abs().max())), (k, fd, float(gc[k]))
    for s, a in ((0, 0), (7, 1), (19, 2)):
        w = X[s, a] - np.floor(X[s, a])
        assert h < w < 1 - h                     # perturbation stays inside the cell
        Xp, Xm = X.copy(), X.copy()
        Xp[s, a] += h
        Xm[s, a] -= h
        fd = (loss_value(p, rho, u, Xp, A, None, coef, n, loss) - loss_value(p, rho, u, Xm, A, None, coef, n, loss)) / (2 * h)
        assert abs(fd - float(gX[s, a])) <= 1e-6 * max(abs(fd), 1e-3 * float(gX.abs().max())), (s, a, fd, float(gX[s, a]))
