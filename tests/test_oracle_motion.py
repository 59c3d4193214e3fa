"""Pins of the oracle's moving solids (prescribed rigid motion, boundary velocity, torque)
against closed forms and physical signs (no GPU)."""
import math

import numpy as np

import scenes
from oracle import motion as mo
from oracle.solver import OracleSolver, Problem


def test_rotation_matrix_is_orthonormal_and_turns_by_the_angle():
    R = mo.rotation((1.0, 2.0, 2.0), 0.7)
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-15 and abs(np.linalg.det(R) - 1) < 1e-15
    k = np.array([1.0, 2.0, 2.0]) / 3.0
    assert np.abs(R @ k - k).max() < 1e-15                      # the axis is fixed
    v = np.array([2.0, -1.0, 0.0]) / math.sqrt(5.0)            # a unit vector normal to the axis
    assert abs(np.dot(R @ v, v) - math.cos(0.7)) < 1e-15
    assert np.abs(np.cross(v, R @ v) - math.sin(0.7) * k).max() < 1e-15   # right-handed


def test_full_turn_and_translation_closed_form():
    X0 = np.array([[12.0, 10.0, 9.0], [10.0, 13.5, 9.0], [10.0, 10.0, 7.0]])
    m = ((10.0, 10.0, 9.0), (0.05, 0.0, -0.02), (0.0, 0.0, 1.0), 2 * math.pi / 40)
    X = mo.sample_positions(X0, m, 40.0)
    assert np.abs(X - (X0 + np.array([2.0, 0.0, -0.8]))).max() < 1e-12
    # a quarter turn about z maps (2, 0, 0) to (0, 2, 0) relative to the centre
    X = mo.sample_positions(X0[:1], m, 10.0)
    assert np.abs(X[0] - np.array([10.0 + 0.5, 12.0, 9.0 - 0.2])).max() < 1e-12


def test_boundary_velocity_is_the_time_derivative_of_the_position():
    X0 = np.random.default_rng(0).uniform(5, 15, (20, 3))
    m = ((10.0, 10.0, 10.0), (0.03, -0.01, 0.02), (1.0, 1.0, 0.0), 0.05)
    tau, h = 3.0, 1e-5
    dX = (mo.sample_positions(X0, m, tau + h) - mo.sample_positions(X0, m, tau - h)) / (2 * h)
    ub = mo.boundary_velocity(mo.sample_positions(X0, m, tau), m, tau)
    assert np.abs(ub - dX).max() < 1e-9


def spinning_sphere(steps, w):
    n = 24
    rho, u = scenes.uniform_flow(n, n, n, (0.0, 0.0, 0.0))
    X, A = scenes.fibonacci_sphere((11.5, 12.0, 12.5), 4.0, 500)
    o = OracleSolver(Problem(n, n, n, nu=0.05))
    o.set_state(rho, u)
    o.set_solids(X, A)
    o.set_motion(((11.5, 12.0, 12.5), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), w))
    o.step(steps)
    return o


def test_spinning_sphere_feels_a_retarding_torque_and_no_net_force():
    """A sphere spun in fluid at rest: the torque about its centre opposes the spin and the
    net force vanishes by symmetry (to the sampling's accuracy)."""
    o = spinning_sphere(6, 0.01)
    T = o.torque((11.5, 12.0, 12.5))
    drag = o.diag["drag"].numpy()
    assert T[2] < 0.0 and abs(T[0]) < 1e-3 * abs(T[2]) and abs(T[1]) < 1e-3 * abs(T[2])
    assert np.abs(drag).max() < 1e-2 * abs(T[2]) / 4.0
    # the spin reverses -> the torque reverses
    assert o.torque((11.5, 12.0, 12.5))[2] == T[2]
    assert spinning_sphere(6, -0.01).torque((11.5, 12.0, 12.5))[2] > 0.0


def test_translating_sphere_feels_drag_against_its_motion():
    n = 24
    rho, u = scenes.uniform_flow(n, n, n, (0.0, 0.0, 0.0))
    X, A = scenes.fibonacci_sphere((9.0, 12.0, 12.0), 3.5, 400)
    o = OracleSolver(Problem(n, n, n, nu=0.05))
    o.set_state(rho, u)
    o.set_solids(X, A)
    V = np.array([0.02, 0.005, 0.0])
    o.set_motion(((9.0, 12.0, 12.0), tuple(V), (0.0, 0.0, 1.0), 0.0))
    o.step(5)
    assert np.dot(o.diag["drag"].numpy(), V) < 0.0
    assert np.abs(o.solids[0].numpy().mean(0) - (np.array([9.0, 12.0, 12.0]) + 4 * V)).max() < 0.05
