"""GPU parity of moving and rotating solids (Algorithm 2 (c): sample update after the IB
stage, torque) against the FP64 oracle.

The device re-poses the samples in FP64 from reference coordinates stored in FP32 relative
to the rotation centre (rounding ~1e-7 of the radius) and rounds the positions to FP32, so
sample positions agree within 1e-5 (|X| < 80: ulp 7.6e-6); everything downstream keeps the
static-solid bars: populations within 3e-7, IB forces within 3e-8 + 1e-6 max|g|, drag and
torque within 1e-5 relative.  The band (a set of nodes) is integer work: its size equals
the number of distinct stencil nodes of the GPU's own positions exactly.
"""
import math

import numpy as np
import pytest

import scenes
from gpu_helpers import compare_populations, lib_solver, need_gpu
from oracle import motion as mo
from oracle.solver import OracleSolver, Problem

pytestmark = pytest.mark.gpu

RATES = dict(omega_bulk=1.3, omega_hi=(1.2, 0.9, 1.45, 1.1))


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def band_size(X, nx, ny):
    b = np.floor(X).astype(np.int64)
    cells = set()
    for d in [(i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]:
        c = b + np.array(d)
        cells.update((c[:, 0] + nx * (c[:, 1] + ny * c[:, 2])).tolist())
    return len(cells)


def run_moving(dims, motion, steps, faces=("periodic",) * 6, u0=(0.0, 0.0, 0.0), u_in=0.0, noise=0.0,
               count=600, radius=3.7, center=None):
    nx, ny, nz = dims
    rho, u = scenes.uniform_flow(nx, ny, nz, u0)
    if center is None:
        center = motion[0]
    X, A = scenes.fibonacci_sphere(center, radius, count)
    g = lib_solver(nx=nx, ny=ny, nz=nz, nu=0.03, faces=faces, u_in=u_in, noise=noise, seed=5, **RATES)
    g.set_state(rho, u)
    g.set_solids(X, A)
    g.set_motion(motion)
    o = OracleSolver(Problem(nx, ny, nz, nu=0.03, faces=tuple(faces), u_in=u_in, noise=noise, seed=5, **RATES))
    o.set_state(rho, u)
    o.set_solids(X, A)
    o.set_motion(motion)
    checks = []
    for t in range(1, steps + 1):
        g.step(1)
        o.step(1)
        Xg = g.solid_samples(count).astype(np.float64)
        Xo = o.solids[0].numpy()
        checks.append((np.abs(Xg - Xo).max(), gpu_band_size(g), band_size(Xg, nx, ny)))
    return g, o, checks


def gpu_band_size(g):
    from paper_2101_11856_gb300 import lbm
    return lbm.lbm_band_size(g.h)


def compare_all(g, o, count, motion, t):
    assert compare_populations(g, o) <= 3e-7
    gg = g.ib_forces(count)
    go = o.diag["g"].numpy().T
    assert np.abs(gg - go).max() <= 3e-8 + 1e-6 * np.abs(go).max()
    _, _, drag_g = g.reductions()
    drag_o = o.diag["drag"].numpy()
    assert np.abs(drag_g - drag_o).max() <= 1e-5 * np.abs(drag_o).max()
    c, _ = mo.pose(motion, t - 1)
    Tg, To = g.torque(), o.torque(c)
    assert np.abs(Tg - To).max() <= 1e-5 * np.abs(To).max(), (Tg, To)
    assert np.abs(g.torque(c) - Tg).max() <= 1e-12 * np.abs(Tg).max() + 1e-15   # NULL centre = current centre


@pytest.mark.parametrize("dims", [(20, 18, 16), (72, 18, 16)])
def test_rotating_translating_sphere_periodic(dims):
    motion = ((8.3, 8.8, 7.9), (0.03, -0.01, 0.015), (0.3, 1.0, 0.5), 0.05)
    g, o, checks = run_moving(dims, motion, 10, u0=(0.02, 0.0, 0.01))
    for dx, nb_g, nb_exact in checks:
        assert dx <= 1e-5
        assert nb_g == nb_exact
    compare_all(g, o, 600, motion, 10)


def test_band_size_matches_after_each_rebuild():
    dims = (40, 30, 28)
    motion = ((14.0, 15.0, 13.0), (0.2, 0.1, -0.05), (0.0, 0.0, 1.0), 0.15)   # fast: the band changes each step
    nx, ny, nz = dims
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.0, 0.0, 0.0))
    X, A = scenes.fibonacci_sphere(motion[0], 5.0, 1500)
    g = lib_solver(nx=nx, ny=ny, nz=nz, nu=0.05)
    g.set_state(rho, u)
    g.set_solids(X, A)
    g.set_motion(motion)
    sizes = set()
    for t in range(12):
        g.step(1)
        Xg = g.solid_samples(1500).astype(np.float64)
        n = gpu_band_size(g)
        assert n == band_size(Xg, nx, ny), t
        sizes.add(n)
    assert len(sizes) > 3


def test_channel_faces_with_moving_sphere():
    dims = (72, 20, 18)
    motion = ((20.0, 10.0, 9.0), (0.04, 0.0, 0.0), (0.0, 1.0, 0.0), -0.03)
    faces = ("inlet", "outlet", "noslip", "noslip", "periodic", "periodic")
    g, o, checks = run_moving(dims, motion, 8, faces=faces, u0=(0.05, 0.0, 0.0), u_in=0.05, noise=0.01, count=500,
                              radius=3.5)
    assert max(c[0] for c in checks) <= 1e-5
    compare_all(g, o, 500, motion, 8)


def test_motion_errors():
    from paper_2101_11856_gb300 import lbm
    n = 16
    rho, u = scenes.uniform_flow(n, n, n, (0.0, 0.0, 0.0))
    g = lib_solver(nx=n, ny=n, nz=n, nu=0.05)
    g.set_state(rho, u)
    with pytest.raises(lbm.LBMError) as e:
        g.set_motion(((8.0, 8.0, 8.0), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 0.1))   # no solid
    assert e.value.code == lbm.LBM_ESTATE
    X, A = scenes.fibonacci_sphere((8.0, 8.0, 8.0), 3.0, 200)
    g.set_solids(X, A)
    g.set_motion(((8.0, 8.0, 8.0), (0.5, 0.0, 0.0), (0.0, 0.0, 1.0), 0.0))        # reaches x = 15 at t = 8
    g.step(7)
    with pytest.raises(lbm.LBMError) as e:
        g.step(3)
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        g.adjoint(2, K=1)
    assert e.value.code == lbm.LBM_EINVAL
    g.set_solids(X, A)                                                          # static again
    g.step(1)
