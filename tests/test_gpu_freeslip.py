"""GPU parity of free-slip y/z faces (half-way specular reflection) against the FP64 oracle,
whose free-slip rule is pinned by the mirror construction (test_oracle_freeslip.py).  Same bars
as the other faces: populations within 2e-7 after a few steps (3e-7 with faces and IB)."""
import numpy as np
import pytest

import scenes
from gpu_helpers import compare_populations, need_gpu, run_pair

pytestmark = pytest.mark.gpu

RATES = dict(omega_bulk=1.3, omega_hi=(1.2, 0.9, 1.45, 1.1))


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("n", [(11, 9, 7), (70, 6, 5), (70, 2, 5), (66, 5, 1)])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_freeslip_box_both_parities(steps, n):
    """(70, 6, 5): face rows and rows off the faces in separate kernels; (70, 2, 5), (66, 5, 1):
    every row on a face."""
    rho, u = scenes.taylor_green(*n, 0.05)
    faces = ("periodic", "periodic", "freeslip", "freeslip", "freeslip", "freeslip")
    g, o = run_pair(*n, 0.03, steps, rho, u, faces=faces, forcing=(1e-5, -2e-5, 3e-5), **RATES)
    assert compare_populations(g, o) <= 2e-7


@pytest.mark.parametrize("dims", [(13, 7, 6), (70, 6, 5), (66, 4, 3)])
@pytest.mark.parametrize("lateral", [("freeslip", "freeslip", "noslip", "noslip"),
                                     ("noslip", "freeslip", "freeslip", "freeslip"),
                                     ("freeslip", "freeslip", "periodic", "periodic")])
def test_channel_corners(dims, lateral):
    """Inlet and outlet x faces against free-slip (and no-slip) lateral faces: every corner rule."""
    nx, ny, nz = dims
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0.0, 0.0))
    coef = scenes.inflow_coefficients(0.004, seed=5)
    faces = ("inlet", "outlet") + tuple(lateral)
    for steps in (1, 2, 25):
        g, o = run_pair(nx, ny, nz, 0.02, steps, rho, u, faces=faces, u_in=0.04, noise=0.01, seed=9,
                        inflow_coef=coef, forcing=(0, -1e-6, 1e-6), **RATES)
        err = compare_populations(g, o)
        assert err <= 3e-7, (steps, err)


def test_sphere_touching_freeslip_walls():
    """IB band nodes on the free-slip face rows (the band-moment pull applies the rule)."""
    nx, ny, nz = 72, 12, 10
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.03, 0.0, 0.0))
    X, A = scenes.fibonacci_sphere((36.2, 2.1, 2.3), 1.9, 200)
    faces = ("periodic", "periodic", "freeslip", "freeslip", "freeslip", "noslip")
    g, o = run_pair(nx, ny, nz, 0.02, 6, rho, u, faces=faces, forcing=(1e-6, 0, 0), samples=X, area=A, **RATES)
    assert compare_populations(g, o) <= 3e-7
    _, _, drag_g = g.reductions()
    _, _, drag_o = o.reductions()
    assert np.abs(drag_g - drag_o.numpy()).max() <= 1e-5 * np.abs(drag_o.numpy()).max()


def test_adjoint_rejects_freeslip():
    from paper_2101_11856_gb300 import lbm
    n = 8
    rho, u = scenes.uniform_flow(n, n, n, (0.0, 0.0, 0.0))
    g, _ = run_pair(n, n, n, 0.05, 0, rho, u, faces=("periodic", "periodic", "freeslip", "freeslip", "periodic",
                                                         "periodic"))
    with pytest.raises(lbm.LBMError) as e:
        g.adjoint(2, K=1)
    assert e.value.code == lbm.LBM_EINVAL


@pytest.mark.parametrize("faces,per_step", [
    (("periodic", "periodic", "freeslip", "noslip", "periodic", "periodic"), {"boundary": 3, "step": 1}),
    (("periodic", "periodic", "noslip", "noslip", "periodic", "periodic"), {"boundary": 1, "step": 1})])
def test_launches_per_step(faces, per_step):
    """A grid with a free-slip face runs its face rows in the boundary part (edge strips of the
    other rows, edge strips and main range of the face rows): the launch counts the library
    reports are those kernels."""
    from paper_2101_11856_gb300 import Solver, lbm
    nx, ny, nz = 80, 6, 5
    rho, u = scenes.taylor_green(nx, ny, nz, 0.03)
    s = Solver(nx, ny, nz, 0.02, faces=faces)
    s.set_state(rho, u)
    lbm.lbm_profile(s.h, True)
    s.step(4)
    kt = lbm.lbm_kernel_times(s.h)
    lbm.lbm_profile(s.h, False)
    s.close()
    for kind, n in per_step.items():
        assert kt[kind][1] == 4 * n, (kind, kt[kind])


def test_many_face_rows_match_periodic():
    """66,000 face rows (more than one grid dimension holds: the row index folds into two).  A
    flow that does not depend on z and has u_z = 0 is symmetric under z -> -z, so free-slip z
    faces give the periodic-z result (y period 60 divides ny)."""
    from paper_2101_11856_gb300 import Solver
    nx, ny, nz = 65, 33000, 2
    y = np.arange(ny, dtype=np.float64)
    x = np.arange(nx, dtype=np.float64)
    ux = 0.03 * np.sin(2 * np.pi * x[None, :] / nx) * np.cos(2 * np.pi * y[:, None] / 60.0)
    uy = 0.02 * np.cos(2 * np.pi * x[None, :] / nx) * np.sin(2 * np.pi * y[:, None] / 60.0)
    u = np.zeros((3, nz, ny, nx), np.float32)
    u[0] = ux[None].astype(np.float32)
    u[1] = uy[None].astype(np.float32)
    rho = np.ones((nz, ny, nx), np.float32)
    out = []
    for zf in ("freeslip", "periodic"):
        # periodic y: the periodic-z run has no free-slip face and runs the kernels without FS
        s = Solver(nx, ny, nz, 0.02, faces=("periodic",) * 4 + (zf, zf))
        s.set_state(rho, u)
        s.step(5)
        out.append(s.populations())
        s.close()
    assert np.abs(out[0] - out[1]).max() <= 1e-6
