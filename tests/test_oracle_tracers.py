"""Pins of the oracle's smoke tracers (advection and density projection) against closed
forms, invariants, the published SplitMix64 vectors and brute force (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import tracers as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EMIT = ((1.0, 2.0, 3.0), (2.0, 6.0, 5.0), 0)


def field(fn, nx, ny, nz):
    """Sample u = fn(x, y, z) on the nodes -> (3, nz, ny, nx)."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack(fn(x.astype(float), y.astype(float), z.astype(float)))


def test_uniform_field_moves_tracers_by_u_with_wrap():
    n = (8, 6, 5)
    c = np.array([0.3, -0.45, 0.2])
    u = field(lambda x, y, z: [c[0] + 0 * x, c[1] + 0 * x, c[2] + 0 * x], *n)
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 1, (50, 3)) * np.array(n)
    X1 = tr.advect(u, X, 1, (True,) * 3, EMIT)
    assert np.abs(X1 - np.mod(X + c, np.array(n))).max() < 1e-12


def test_linear_field_midpoint_closed_form():
    """Trilinear interpolation is exact for a linear field, so one step is
    x' = x + A (x + (A x + b)/2) + b exactly (the explicit midpoint rule)."""
    n = (12, 10, 9)
    A = np.array([[0.01, -0.02, 0.005], [0.015, 0.0, -0.01], [-0.005, 0.02, 0.01]])
    b = np.array([0.05, -0.03, 0.02])
    u = field(lambda x, y, z: [A[i, 0] * x + A[i, 1] * y + A[i, 2] * z + b[i] for i in range(3)], *n)
    rng = np.random.default_rng(1)
    X = rng.uniform(2, 6, (40, 3))
    assert np.abs(tr.interpolate(u, X, (False,) * 3) - (X @ A.T + b)).max() < 1e-13
    Xm = X + 0.5 * (X @ A.T + b)
    expect = X + Xm @ A.T + b
    assert np.abs(tr.advect(u, X, 1, (False,) * 3, EMIT) - expect).max() < 1e-13


def test_rotation_growth_and_phase_of_the_midpoint_rule():
    """Solid rotation u = w e_z x (x - c): the midpoint rule multiplies the radius by
    sqrt(1 + w^4/4) and advances the angle by atan2(w, 1 - w^2/2) per step (an Euler step
    would give sqrt(1 + w^2) and atan(w))."""
    n = (40, 40, 3)
    w, c = 0.05, np.array([20.0, 20.0])
    u = field(lambda x, y, z: [-w * (y - c[1]), w * (x - c[0]), 0 * x], *n)
    X = np.array([[28.0, 20.0, 1.0]])
    steps = 20
    for t in range(steps):
        X = tr.advect(u, X, t + 1, (False, False, True), EMIT)
    r = math.hypot(X[0, 0] - c[0], X[0, 1] - c[1])
    theta = math.atan2(X[0, 1] - c[1], X[0, 0] - c[0])
    assert abs(r - 8.0 * (1 + w ** 4 / 4) ** (steps / 2)) < 1e-11
    assert abs(theta - steps * math.atan2(w, 1 - w * w / 2)) < 1e-12


def test_reinjection_uses_the_published_splitmix64_outputs():
    """Tracer 0 of 1 leaving through +x at step 1 draws counters 0, 1, 2 of seed 0."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if not l.startswith("#")]
    outs = [int(v, 16) for s, n, v in rows if s == "0"]
    U = np.array([(o >> 40) * 2.0 ** -24 for o in outs])
    n = (6, 8, 7)
    u = field(lambda x, y, z: [0.4 + 0 * x, 0 * x, 0 * x], *n)
    lo, hi = np.array(EMIT[0]), np.array(EMIT[1])
    X1 = tr.advect(u, np.array([[4.8, 3.0, 3.0]]), 1, (False,) * 3, EMIT)
    assert np.abs(X1[0] - (lo + (hi - lo) * U)).max() < 1e-15
    # a tracer that stays inside is not re-injected
    X2 = tr.advect(u, np.array([[4.5, 3.0, 3.0]]), 1, (False,) * 3, EMIT)
    assert abs(X2[0, 0] - 4.9) < 1e-12


def test_midpoint_outside_triggers_reinjection():
    n = (6, 8, 7)
    u = field(lambda x, y, z: [0 * x, -0.6 + 0 * x, 0 * x], *n)   # midpoint y = 0.1 - 0.3 < 0
    X1 = tr.advect(u, np.array([[2.0, 0.1, 3.0]]), 1, (False,) * 3, EMIT)
    lo, hi = np.array(EMIT[0]), np.array(EMIT[1])
    assert np.all(X1[0] >= lo) and np.all(X1[0] < hi)


def brute_density(X, shape_xyz, periodic, s):
    """Every voxel v sums prod_a hat(d_a) over tracers, d the (wrapped) offset in voxels."""
    dims = tr.grid_dims(shape_xyz, periodic, s)
    rho = np.zeros(dims[::-1])
    for p in X / s:
        for v in np.ndindex(*dims[::-1]):
            wgt = 1.0
            for a in range(3):
                d = p[a] - v[2 - a]
                if periodic[a]:
                    d = (d + dims[a] / 2) % dims[a] - dims[a] / 2
                wgt *= max(0.0, 1.0 - abs(d))
            rho[v] += wgt
    return rho


@pytest.mark.parametrize("periodic", [(True, True, True), (False, False, True), (False, False, False)])
@pytest.mark.parametrize("s", [1, 2])
def test_density_brute_force_mass_and_first_moment(periodic, s):
    shape = (8, 6, 4)
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, (25, 3)) * (np.array(shape) - np.where(periodic, 0, 1))
    X[0] = [0.0, 0.0, 0.0]
    X[1] = [shape[0] - 1.0 if not periodic[0] else 7.5, 2.0, 1.0]
    rho = tr.density(X, shape, periodic, s)
    assert np.abs(rho - brute_density(X, shape, periodic, s)).max() < 1e-12
    assert abs(rho.sum() - X.shape[0]) < 1e-12
    gz, gy, gx = rho.shape
    for a, g in enumerate((gx, gy, gz)):
        if not periodic[a]:
            coord = np.arange(g) * s
            m = np.tensordot(rho.sum(tuple(i for i in range(3) if i != 2 - a)), coord, 1)
            assert abs(m - X[:, a].sum()) < 1e-10


def test_density_node_and_top_face():
    shape = (5, 5, 5)
    X = np.array([[2.0, 3.0, 1.0], [4.0, 4.0, 4.0]])
    rho = tr.density(X, shape, (False,) * 3, 1)
    assert rho[1, 3, 2] == 1.0 and rho[4, 4, 4] == 1.0 and rho.sum() == 2.0
