"""GPU parity of the comparison collision models of Sec. 6.1 (D3Q27 BGK and raw-moment MRT)
against the FP64 oracle, under the same streaming, faces, Guo forcing and immersed
boundary as the ACM-MRT step.  Same bars as the ACM-MRT parity tests: populations after a
few steps within 2e-7 (3e-7 with faces and IB), rho and u within 1e-5 relative L2 after 100
steps."""
import numpy as np
import pytest

import scenes
from gpu_helpers import compare_fields, compare_populations, need_gpu, run_pair

pytestmark = pytest.mark.gpu

RATES = dict(omega_bulk=1.3, omega_hi=(1.2, 0.9, 1.45, 1.1))
MODELS = ("bgk", "raw")


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("n", [(11, 9, 7), (70, 5, 4)])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_populations_both_aa_parities(model, steps, n):
    rho, u = scenes.taylor_green(*n, 0.05)
    g, o = run_pair(*n, 0.03, steps, rho, u, forcing=(1e-5, -2e-5, 3e-5), collision=model, **RATES)
    err = compare_populations(g, o)
    assert err <= 2e-7, err


# BGK relaxes every non-conserved moment at omega_s = 1.887 (nu = 0.01), so the FP32 rounding
# of each step's equilibrium is over-relaxed and decays only by |1 - omega_s| = 0.887 per step
# instead of being reset by the omega ~ 1 rates of the higher moments; the BGK update
# evaluated in FP32 numpy arithmetic on this case (FP64 streaming, FP32 collision) drifts to
# 1.0e-5 relative L2 in j after 100 steps.  The BGK bar is 3x that; the MRT models keep 1e-5.
TGV_U_BAR = {"bgk": 3e-5, "raw": 1e-5}


@pytest.mark.parametrize("model", MODELS)
def test_tgv_100_steps(model):
    dims = (96, 10, 12)
    rho, u = scenes.taylor_green(*dims, 0.05)
    g, o = run_pair(*dims, 0.01, 100, rho, u, collision=model, **RATES)
    e_rho, _, e_u = compare_fields(g, o)
    print(f"{model} TGV {dims} 100 steps: rel L2 rho {e_rho:.2e}, u {e_u:.2e}")
    assert e_rho <= 1e-5 and e_u <= TGV_U_BAR[model]


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("dims", [(13, 7, 9), (77, 6, 5)])
def test_channel_faces(model, dims):
    nx, ny, nz = dims
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0.0, 0.0))
    coef = scenes.inflow_coefficients(0.004, seed=5)
    faces = ("inlet", "outlet", "noslip", "noslip", "periodic", "periodic")
    g, o = run_pair(nx, ny, nz, 0.02, 25, rho, u, faces=faces, u_in=0.04, noise=0.01, seed=9, inflow_coef=coef,
                    forcing=(0, -1e-6, 0), collision=model, **RATES)
    assert compare_populations(g, o) <= 3e-7


@pytest.mark.parametrize("model", MODELS)
def test_immersed_sphere(model):
    nx, n = 72, 16
    rho, u = scenes.taylor_green(nx, n, n, 0.04)
    X, A = scenes.fibonacci_sphere((33.3, 8.1, 6.6), 3.7, 300)
    ub = np.tile([0.01, -0.005, 0.0], (300, 1))
    g, o = run_pair(nx, n, n, 0.02, 6, rho, u, forcing=(1e-6, 0, 0), samples=X, area=A, u_b=ub, collision=model,
                    **RATES)
    assert compare_populations(g, o) <= 3e-7
    _, _, drag_g = g.reductions()
    _, _, drag_o = o.reductions()
    assert np.abs(drag_g - drag_o.numpy()).max() <= 1e-5 * np.abs(drag_o.numpy()).max()


@pytest.mark.parametrize("model", MODELS)
def test_fp16_storage_runs(model):
    s = scenes.scene_tgv32()
    g, o = run_pair(32, 32, 32, s["nu"], 50, s["rho"], s["u"], storage="f16", collision=model)
    _, _, e_u = compare_fields(g, o)
    print(f"{model} f16 TGV32 50 steps: rel L2 u {e_u:.2e}")
    assert np.isfinite(e_u) and e_u <= 5e-3


@pytest.mark.parametrize("model", MODELS)
def test_adjoint_is_acm_only(model):
    from paper_2101_11856_gb300 import lbm
    rho, u = scenes.taylor_green(8, 8, 8, 0.02)
    g, _ = run_pair(8, 8, 8, 0.05, 0, rho, u, collision=model)
    with pytest.raises(lbm.LBMError) as e:
        g.adjoint(2, K=1)
    assert e.value.code == lbm.LBM_EINVAL
