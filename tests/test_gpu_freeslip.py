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


@pytest.mark.parametrize("n", [(11, 9, 7), (70, 6, 5)])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_freeslip_box_both_parities(steps, n):
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
