"""GPU tests of the C ABI's contract: argument and state errors, host/device pointers,
checkpoints, solid replacement, degenerate grids, instability and wait limits."""
import numpy as np
import pytest
import torch

import scenes
from gpu_helpers import compare_fields, compare_populations, need_gpu, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def make(n=8, **kw):
    from paper_2101_11856_gb300 import Solver
    s = Solver(n, n, n, 0.05, **kw)
    return s


def test_step_before_state_is_a_state_error():
    from paper_2101_11856_gb300 import LBMError, lbm
    s = make()
    with pytest.raises(LBMError) as e:
        s.step(1)
    assert e.value.code == lbm.LBM_ESTATE


def test_invalid_samples_rejected_and_previous_solid_kept():
    from paper_2101_11856_gb300 import LBMError, lbm
    s = make(10)
    rho, u = scenes.taylor_green(10, 10, 10, 0.02)
    s.set_state(rho, u)
    X, A = scenes.fibonacci_sphere((4.5, 4.5, 4.5), 2.0, 50)
    s.set_solids(X, A)
    nb = lbm.lbm_band_size(s.h)
    assert nb > 0
    for bad in (np.array([[9.0, 1.0, 1.0]]), np.array([[-0.1, 1.0, 1.0]]), np.array([[1.0, np.nan, 1.0]])):
        with pytest.raises(LBMError) as e:
            s.set_solids(bad)
        assert e.value.code == lbm.LBM_EINVAL
        assert lbm.lbm_band_size(s.h) == nb
    s.set_solids(None)                       # count = 0 removes the solid
    assert lbm.lbm_band_size(s.h) == 0
    s.step(2)
    assert lbm.lbm_check(s.h) == lbm.LBM_OK


def test_zero_steps_and_time_counter():
    s = make()
    rho, u = scenes.taylor_green(8, 8, 8, 0.02)
    s.set_state(rho, u)
    r0, u0 = s.macroscopic()
    s.step(0)
    assert s.time == 0
    r1, u1 = s.macroscopic()
    assert np.array_equal(r0, r1) and np.array_equal(u0, u1)
    assert np.abs(u0 - u).max() < 1e-7 and np.abs(r0 - rho).max() < 1e-6
    s.step(3)
    assert s.time == 3


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_checkpoint_roundtrip_is_bit_exact(storage):
    from paper_2101_11856_gb300 import LBMError, Solver, lbm
    kw = dict(faces=("inlet", "outlet", "noslip", "noslip", "periodic", "periodic"), u_in=0.03, noise=0.01,
              storage=storage)
    s = make(12, **kw)
    rho, u = scenes.uniform_flow(12, 12, 12, (0.03, 0, 0))
    s.set_state(rho, u)
    X, A = scenes.fibonacci_sphere((5.5, 6.0, 6.0), 2.5, 80)
    s.set_solids(X, A)
    s.step(5)
    blob = lbm.lbm_save(s.h)
    s.step(5)
    fa = s.populations()
    lbm.lbm_load(s.h, blob)
    assert s.time == 5
    s.step(5)
    fb = s.populations()
    assert np.array_equal(fa, fb)
    other = make(10)
    with pytest.raises(Exception):
        lbm.lbm_load(other.h, blob)
    # same dims and storage under another configuration: refused, the state is kept
    for change in (dict(nu=0.06), dict(u_in=0.04), dict(noise=0.02), dict(omega_hi=(1.0, 1.2, 1.0, 1.0))):
        kw2 = dict(kw, **{k: v for k, v in change.items() if k != "nu"})
        o2 = Solver(12, 12, 12, change.get("nu", 0.05), **kw2)
        o2.set_state(rho, u)
        o2.step(1)
        with pytest.raises(LBMError) as e:
            lbm.lbm_load(o2.h, blob)
        assert e.value.code == lbm.LBM_EINVAL and o2.time == 1, change
        o2.close()


def test_per_sample_outputs_take_their_length_from_the_context():
    """adjoint() and ib_forces() with default arguments return one row per installed sample;
    a count that differs from the context's is refused before the library writes anything."""
    from paper_2101_11856_gb300 import lbm
    n = 12
    s = make(n, faces=("inlet", "outlet", "periodic", "periodic", "periodic", "periodic"), u_in=0.03)
    s.set_state(*scenes.uniform_flow(n, n, n, (0.03, 0, 0)))
    X, A = scenes.fibonacci_sphere((5.5, 6.0, 6.0), 2.5, 80)
    s.set_solids(X, A)
    assert lbm.lbm_solid_count(s.h) == 80 and lbm.lbm_dims(s.h) == (n, n, n)
    L, dc, dx = s.adjoint(3, 2)
    assert dx.shape == (80, 3) and np.all(np.isfinite(dx)) and np.isfinite(L)
    assert s.ib_forces().shape == (80, 3)
    for bad in (0, 79, 81):
        with pytest.raises(ValueError):
            s.adjoint(2, 1, count=bad)
        with pytest.raises(ValueError):
            s.ib_forces(bad)
    with pytest.raises(ValueError):
        lbm.lbm_ib_forces(s.h, np.empty((79, 3), np.float32))
    with pytest.raises(ValueError):
        lbm.lbm_macroscopic(s.h, np.empty(n ** 3, np.float64), None)
    s.set_solids(None)
    L, dc, dx = s.adjoint(2, 1)
    assert dx.shape == (0, 3)
    s.close()


def test_device_and_host_pointers_agree():
    from paper_2101_11856_gb300 import lbm
    n = 10
    rho, u = scenes.taylor_green(n, n, n, 0.04)
    a = make(n)
    a.set_state(rho, u)
    b = make(n)
    b.set_state(torch.tensor(rho, dtype=torch.float32, device="cuda"), torch.tensor(u, dtype=torch.float32, device="cuda"))
    a.step(4)
    b.step(4)
    rh, uh = a.macroscopic()
    rd = torch.empty(n ** 3, device="cuda")
    ud = torch.empty(3, n ** 3, device="cuda")
    lbm.lbm_macroscopic(b.h, rd, ud)
    torch.cuda.synchronize()
    assert np.array_equal(rh.ravel(), rd.cpu().numpy())
    assert np.array_equal(uh.reshape(3, -1), ud.cpu().numpy())


def test_nan_state_is_detected():
    from paper_2101_11856_gb300 import lbm
    rho, u = scenes.taylor_green(8, 8, 8, 0.02)
    rho[3, 4, 5] = np.nan
    s = make()
    s.set_state(rho, u)
    s.step(2)
    assert lbm.lbm_check(s.h) == lbm.LBM_EUNSTABLE
    good = make()
    good.set_state(*scenes.taylor_green(8, 8, 8, 0.02))
    good.step(2)
    assert lbm.lbm_check(good.h) == lbm.LBM_OK


def test_synchronize_wall_clock_limit():
    """A bounded GPU sleep on the context's stream outlasts a 20 ms wait limit."""
    from paper_2101_11856_gb300 import LBMError, lbm
    s = make()
    s.set_state(*scenes.taylor_green(8, 8, 8, 0.02))
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2e9))              # ~1 s of device time, then it ends by itself
    with pytest.raises(LBMError) as e:
        lbm.lbm_synchronize(s.h, 0.02)
    assert e.value.code == lbm.LBM_ETIMEOUT
    lbm.lbm_synchronize(s.h, 30.0)


@pytest.mark.parametrize("dims,faces", [
    ((1, 6, 1), ("periodic", "periodic", "noslip", "noslip", "periodic", "periodic")),
    ((2, 3, 2), ("periodic",) * 6),
    ((3, 3, 3), ("inlet", "outlet", "noslip", "noslip", "noslip", "noslip")),
    ((5, 1, 4), ("inlet", "outlet", "periodic", "periodic", "periodic", "periodic")),
])
def test_degenerate_grids(dims, faces):
    """Grids with no interior cells run entirely through the face-cell kernel."""
    nx, ny, nz = dims
    rho, u = scenes.taylor_green(nx, ny, nz, 0.02) if "inlet" not in faces else scenes.uniform_flow(nx, ny, nz, (0.02, 0, 0))
    g, o = run_pair(nx, ny, nz, 0.05, 4, rho, u, faces=faces, u_in=0.02, forcing=(1e-5, 0, 0))
    assert compare_populations(g, o) <= 2e-7
