"""GPU adjoint (through the C ABI) against the FP64 oracle's reverse-mode gradients.

The oracle's gradients are pinned to central finite differences (test_oracle_adjoint.py);
here the FP32 hand-written adjoint must match them: loss to 1e-5 relative, gradient vectors
to 1e-3 relative L2 (FP32 arithmetic in forward and backward over a few steps)."""
import numpy as np
import pytest
import torch

import scenes
from gpu_helpers import need_gpu, rel_l2
from oracle.adjoint import Loss, loss_and_gradients
from oracle.solver import Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def run_both(nx, ny, nz, nu, n, K, loss, faces, rho, u, X=None, A=None, ub=None, coef=None, u_in=0.0, noise=0.0,
             forcing=(0.0, 0.0, 0.0), rates=None):
    from paper_2101_11856_gb300 import Solver
    rates = rates or dict(omega_bulk=1.0, omega_hi=(1.0, 1.0, 1.0, 1.0))
    s = Solver(nx, ny, nz, nu, forcing=forcing, faces=faces, u_in=u_in, noise=noise, seed=11, inflow_coef=coef, **rates)
    s.set_state(rho, u)
    count = 0
    if X is not None:
        s.set_solids(X, A, ub)
        count = len(X)
    Lg, dcg, dxg = s.adjoint(n, K, loss.w_drag, loss.w_ke, loss.ke_x0, loss.ke_x1, count)
    p = Problem(nx, ny, nz, nu=nu, forcing=forcing, faces=faces, u_in=u_in, noise=noise, seed=11,
                omega_bulk=rates["omega_bulk"], omega_hi=tuple(rates["omega_hi"]))
    c = np.zeros(16) if coef is None else coef
    Xo = np.zeros((0, 3)) if X is None else X.astype(np.float32).astype(np.float64)
    Lo, dco, dxo = loss_and_gradients(p, rho, u, Xo, A, ub, c, n, loss) if X is not None else (None, None, None)
    return s, (Lg, dcg, dxg), (Lo, dco, dxo)


def test_channel_sphere_drag_and_ke_with_segments():
    nx, ny, nz = 14, 8, 8
    faces = ("inlet", "outlet", "periodic", "periodic", "periodic", "periodic")
    X, A = scenes.fibonacci_sphere((5.3, 3.6, 3.4), 1.7, 24)
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0, 0))
    coef = np.random.default_rng(1).uniform(-0.005, 0.005, 16)
    loss = Loss(1.0, 2.0, 10, 13)
    for K in (6, 4, 1):
        s, (Lg, dcg, dxg), (Lo, dco, dxo) = run_both(nx, ny, nz, 0.05, 6, K, loss, faces, rho, u, X, A, coef=coef,
                                                     u_in=0.04, noise=0.01)
        print(f"K={K}: L {Lg:.6e} vs {Lo:.6e}; rel dtheta {rel_l2(dcg, dco.numpy()):.2e}; rel dX {rel_l2(dxg, dxo.numpy()):.2e}")
        assert abs(Lg - Lo) <= 1e-5 * abs(Lo)
        assert rel_l2(dcg, dco.numpy()) <= 1e-3
        assert rel_l2(dxg, dxo.numpy()) <= 1e-3
        assert s.time == 6


def test_periodic_box_forced_distinct_rates():
    n = 10
    rho, u = scenes.taylor_green(n, n, n, 0.04)
    X, A = scenes.fibonacci_sphere((4.6, 5.2, 4.9), 2.4, 40)
    ub = np.tile([0.01, -0.005, 0.002], (40, 1))
    rates = dict(omega_bulk=1.3, omega_hi=(1.2, 0.9, 1.45, 1.1))
    loss = Loss(1.0, 0.5, 2, 7)
    s, (Lg, dcg, dxg), (Lo, dco, dxo) = run_both(n, n, n, 0.03, 5, 2, loss, ("periodic",) * 6, rho, u, X, A, ub,
                                                 forcing=(1e-5, -2e-5, 0), rates=rates)
    print(f"L {Lg:.6e} vs {Lo:.6e}; rel dX {rel_l2(dxg, dxo.numpy()):.2e}")
    assert abs(Lg - Lo) <= 1e-5 * abs(Lo)
    assert rel_l2(dxg, dxo.numpy()) <= 1e-3
    assert np.all(dcg == 0.0)


def test_noslip_walls_outlet_ke_only():
    nx, ny, nz = 12, 7, 6
    faces = ("inlet", "outlet", "noslip", "noslip", "noslip", "noslip")
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.03, 0, 0))
    X, A = scenes.fibonacci_sphere((4.5, 3.1, 2.6), 1.2, 12)
    coef = np.random.default_rng(2).uniform(-0.004, 0.004, 16)
    loss = Loss(0.0, 1.0, 6, 12)
    s, (Lg, dcg, dxg), (Lo, dco, dxo) = run_both(nx, ny, nz, 0.04, 7, 3, loss, faces, rho, u, X, A, coef=coef,
                                                 u_in=0.03)
    print(f"L {Lg:.6e} vs {Lo:.6e}; rel dtheta {rel_l2(dcg, dco.numpy()):.2e}; rel dX {rel_l2(dxg, dxo.numpy()):.2e}")
    assert abs(Lg - Lo) <= 1e-5 * abs(Lo)
    assert rel_l2(dcg, dco.numpy()) <= 1e-3
    assert rel_l2(dxg, dxo.numpy()) <= 1e-3


def test_adjoint_advances_state_like_forward_steps():
    from paper_2101_11856_gb300 import Solver
    nx, ny, nz = 16, 9, 8
    faces = ("inlet", "outlet", "periodic", "periodic", "noslip", "noslip")
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0, 0))
    X, A = scenes.fibonacci_sphere((6.0, 4.2, 3.7), 2.0, 30)
    a = Solver(nx, ny, nz, 0.04, faces=faces, u_in=0.04, noise=0.01)
    b = Solver(nx, ny, nz, 0.04, faces=faces, u_in=0.04, noise=0.01)
    for s in (a, b):
        s.set_state(rho, u)
        s.set_solids(X, A)
    a.adjoint(7, 3, 1.0, 1.0, 8, 16, 30)
    b.step(7)
    assert np.array_equal(a.populations(), b.populations())
    assert np.allclose(a.reductions()[2], b.reductions()[2], rtol=0, atol=0)


@pytest.mark.parametrize("K", [4, 2, 1])
def test_long_rows_main_and_edge_kernels(K):
    """nx = 70: the backward main kernel takes 1 <= x <= 68 in two 64-node chunks per row (the
    lanes past nx - 2 idle) and the x-face kernel the two end nodes, against the oracle; K = 2
    keeps all three segments from the forward pass (up to four segment sets fit), K = 1 keeps the
    last four and recomputes the first two on the second stream.  The sphere lies in the main
    range, the kinetic-energy slab next to the inlet (so that the inflow coefficients reach the
    loss within the 6 steps)."""
    nx, ny, nz = 70, 6, 5
    faces = ("inlet", "outlet", "noslip", "noslip", "periodic", "periodic")
    X, A = scenes.fibonacci_sphere((37.4, 2.6, 2.3), 1.6, 30)
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0, 0))
    coef = np.random.default_rng(3).uniform(-0.004, 0.004, 16)
    loss = Loss(1.0, 1.5, 1, 5)
    s, (Lg, dcg, dxg), (Lo, dco, dxo) = run_both(nx, ny, nz, 0.04, 6, K, loss, faces, rho, u, X, A, coef=coef,
                                                 u_in=0.04, noise=0.01,
                                                 rates=dict(omega_bulk=1.2, omega_hi=(1.1, 0.95, 1.3, 1.05)))
    print(f"nx=70 K={K}: L {Lg:.6e} vs {Lo:.6e}; rel dtheta {rel_l2(dcg, dco.numpy()):.2e}; "
          f"rel dX {rel_l2(dxg, dxo.numpy()):.2e}")
    assert abs(Lg - Lo) <= 1e-5 * abs(Lo)
    assert np.abs(dco.numpy()).max() > 0 and np.abs(dxo.numpy()).max() > 0
    assert rel_l2(dcg, dco.numpy()) <= 1e-3
    assert rel_l2(dxg, dxo.numpy()) <= 1e-3


@pytest.mark.parametrize("where", ["inlet", "outlet"])
def test_band_at_the_x_faces(where):
    """A sphere whose band reaches x = 0 (next to the inlet) or x = nx - 1 (next to the outlet):
    band nodes in the x-face kernel (with the inlet's bounce-back and inflow gradient, or the
    outlet ghost's second use), against the oracle; K = 2 with 6 steps recomputes one segment."""
    nx, ny, nz = 16, 8, 8
    faces = ("inlet", "outlet", "periodic", "periodic", "noslip", "noslip")
    cx = 1.9 if where == "inlet" else nx - 2.7
    X, A = scenes.fibonacci_sphere((cx, 3.6, 3.4), 1.2, 20)
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0, 0))
    coef = np.random.default_rng(5).uniform(-0.004, 0.004, 16)
    loss = Loss(1.0, 1.5, 4, 9)
    s, (Lg, dcg, dxg), (Lo, dco, dxo) = run_both(nx, ny, nz, 0.04, 6, 2, loss, faces, rho, u, X, A, coef=coef,
                                                 u_in=0.04, noise=0.01)
    print(f"band at the {where}: L {Lg:.6e} vs {Lo:.6e}; rel dtheta {rel_l2(dcg, dco.numpy()):.2e}; "
          f"rel dX {rel_l2(dxg, dxo.numpy()):.2e}")
    assert abs(Lg - Lo) <= 1e-5 * abs(Lo)
    assert rel_l2(dcg, dco.numpy()) <= 1e-3
    assert rel_l2(dxg, dxo.numpy()) <= 1e-3


def test_long_rows_periodic_box():
    nx, ny, nz = 72, 6, 6
    rho, u = scenes.taylor_green(nx, ny, nz, 0.04)
    X, A = scenes.fibonacci_sphere((33.3, 3.1, 2.8), 1.8, 30)
    ub = np.tile([0.01, 0.0, -0.004], (30, 1))
    loss = Loss(1.0, 0.7, 30, 42)
    s, (Lg, dcg, dxg), (Lo, dco, dxo) = run_both(nx, ny, nz, 0.03, 5, 3, loss, ("periodic",) * 6, rho, u, X, A, ub,
                                                 forcing=(1e-5, 0, -1e-5))
    print(f"nx=72 periodic: L {Lg:.6e} vs {Lo:.6e}; rel dX {rel_l2(dxg, dxo.numpy()):.2e}")
    assert abs(Lg - Lo) <= 1e-5 * abs(Lo)
    assert rel_l2(dxg, dxo.numpy()) <= 1e-3


def test_c5_fullsize_directional_derivatives():
    """The adjoint workload at full size (128^3 channel, 2,000-sample sphere, 200 steps, K = 20,
    loss = mean drag + kinetic energy of 96 <= x < 128, gradients at a = 0): the loss's
    central differences along the adjoint's own gradient directions equal the gradient
    norms.  Inflow coefficients: step 1e-3 (the loss is smooth in a), bar 1e-4; positions:
    step 1e-2 cells (the trilinear weights have kinks at cell faces, and the FP32 loss of ~660
    has ~1e-4 noise), bar 3 %."""
    from paper_2101_11856_gb300 import Solver
    n = 128
    X, A = scenes.fibonacci_sphere((40.0, 64, 64), 12.6, 2000)
    rho, u = scenes.uniform_flow(n, n, n, (0.05, 0, 0))
    s = Solver(n, n, n, 0.01, faces=("inlet", "outlet", "periodic", "periodic", "periodic", "periodic"),
               u_in=0.05, noise=0.01, seed=2101)

    def run(coef, Xs):
        s.set_inflow(coef)
        s.set_solids(Xs.astype(np.float32), A)
        s.set_state(rho, u)
        return s.adjoint(200, 20, 1.0, 1.0, 96, 128, 2000)

    a0 = np.zeros(16)
    L, dc, dx = run(a0, X)
    e = dc / np.linalg.norm(dc)
    fd_c = (run(a0 + 1e-3 * e, X)[0] - run(a0 - 1e-3 * e, X)[0]) / 2e-3
    ex = dx / np.linalg.norm(dx)
    fd_x = (run(a0, X + 1e-2 * ex)[0] - run(a0, X - 1e-2 * ex)[0]) / 2e-2
    print(f"C5: L {L:.4f}; |dL/da| {np.linalg.norm(dc):.6e} vs {fd_c:.6e}; |dL/dX| {np.linalg.norm(dx):.5e} vs {fd_x:.5e}")
    assert abs(fd_c - np.linalg.norm(dc)) <= 1e-4 * np.linalg.norm(dc)
    assert abs(fd_x - np.linalg.norm(dx)) <= 3e-2 * np.linalg.norm(dx)
