"""Moving and rotating solids: prescribed rigid motion of the solid samples, their boundary
velocity, and the torque on the solid (Algorithm 2 (c): after the penalty forces are
spread, the total force and torque are reduced and the solid samples are updated; the
paper's dynamic solids are a rotating torus and a moving airplane, Sec. 6).

ORACLE -- test infrastructure only.

Readings (the paper prints no formulas for the update):

* A motion is (c0, V, a, w): the samples given to ``set_solids`` are the pose at time 0,
  c0 the rotation centre of that pose, V the translation per step, a the rotation axis
  (normalised here) and w the angular velocity in radians per step.  The pose at time tau
  is c(tau) = c0 + V tau and R(tau) = the rotation by the angle w tau about a (Rodrigues'
  formula), and a sample with reference position X0 sits at c(tau) + R(tau) (X0 - c0).
* Step t (1-based) runs its immersed-boundary stage with the samples at the pose of time
  t - 1: the update of Algorithm 2 that follows the IB stage of step t - 1.  The boundary
  velocity of a sample is the rigid-body velocity u_b = V + w a x (X - c(t - 1)).
* Torque on the solid about a centre c: T = sum_s (X_s - c) x (-g_s), with -g_s the force
  of the fluid on the solid at sample s (the drag is -sum g_s).
"""
from __future__ import annotations

import math

import numpy as np


def rotation(axis, angle: float) -> np.ndarray:
    """Rotation matrix by ``angle`` about ``axis`` (Rodrigues' formula)."""
    k = np.asarray(axis, dtype=np.float64)
    n = np.linalg.norm(k)
    if n == 0.0 or angle == 0.0:
        return np.eye(3)
    k = k / n
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def pose(motion, tau: float):
    """(centre, rotation matrix) at time tau; motion = (c0, V, axis, w)."""
    c0, V, axis, w = motion
    return np.asarray(c0, dtype=np.float64) + np.asarray(V, dtype=np.float64) * tau, rotation(axis, w * tau)


def sample_positions(X0: np.ndarray, motion, tau: float) -> np.ndarray:
    """Positions (S, 3) of the reference samples X0 (S, 3) at time tau."""
    c, R = pose(motion, tau)
    return c + (X0 - np.asarray(motion[0], dtype=np.float64)) @ R.T


def boundary_velocity(X: np.ndarray, motion, tau: float) -> np.ndarray:
    """Rigid-body velocity (S, 3) of the samples X at time tau."""
    c0, V, axis, w = motion
    c, _ = pose(motion, tau)
    k = np.asarray(axis, dtype=np.float64)
    n = np.linalg.norm(k)
    Om = w * k / n if n > 0.0 else np.zeros(3)
    return np.asarray(V, dtype=np.float64) + np.cross(Om, X - c)


def torque(X: np.ndarray, g: np.ndarray, center) -> np.ndarray:
    """Torque on the solid about ``center``: sum_s (X_s - c) x (-g_s); X, g (S, 3)."""
    return np.cross(X - np.asarray(center, dtype=np.float64), -g).sum(0)
