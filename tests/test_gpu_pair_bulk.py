"""The tensor-copy fed main kernel for 16-bit storage (k_step_pair_tma, lbm_set_pair_kernel(h, 1)):
its CTAs stage each row tile's 27 source segments in shared memory with tiled tensor copies
(cp.async.bulk.tensor) and collide the node pairs from there.  It reads the same stored values and runs the same
FP32 arithmetic as the register-fed pair kernel (pinned against the FP64 oracle by
test_gpu_precision.py and test_gpu_parity.py), so every result must be bit-identical to it: on
rows away from the y/z faces, on wrapped and bounced face rows, with the free-slip face rows in
their own kernels, with a solid, with the velocity output of the smoke tracers, for tiles cut
short at the end of a row, over batches of steps of both AA parities."""
import numpy as np
import pytest

import scenes
from gpu_helpers import lib_solver, need_gpu

pytestmark = pytest.mark.gpu

RATES = dict(omega_bulk=1.3, omega_hi=(1.2, 0.9, 1.45, 1.1))
CITY_FACES = ("inlet", "outlet", "noslip", "freeslip", "periodic", "periodic")


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _run(bulk, dims, faces, storage, batches, solid=None, tracers=False, u0=(0.04, 0.0, 0.0), rho_noise=0.0):
    nx, ny, nz = dims
    s = lib_solver(nx=nx, ny=ny, nz=nz, nu=0.02, forcing=(1e-6, -2e-6, 3e-6), storage=storage, faces=faces,
                   u_in=0.04, noise=0.01, seed=13, **RATES)
    s.set_pair_kernel(bulk)
    rho, u = scenes.uniform_flow(nx, ny, nz, u0)
    if rho_noise:
        rng = np.random.default_rng(4)
        rho = (rho + rho_noise * rng.standard_normal(rho.shape)).astype(np.float32)
        u = (u + rho_noise * rng.standard_normal(u.shape)).astype(np.float32)
    s.set_state(rho, u)
    if solid is not None:
        s.set_solids(*solid)
    if tracers:
        rng = np.random.default_rng(3)
        s.set_tracers((rng.uniform(0, 1, (400, 3)) * np.array([nx - 1, ny - 1, nz - 1])).astype(np.float32),
                      ((1.0, 1.0, 1.0), (6.0, ny - 2.0, nz - 2.0), 7))
    for n in batches:
        s.step(n)
    return s


def _same(a, b):
    fa, fb = a.populations(), b.populations()
    assert np.array_equal(fa, fb), float(np.abs(fa - fb).max())
    ra, ua = a.macroscopic()
    rb, ub = b.macroscopic()
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
    assert a.reductions()[0] == b.reductions()[0]


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("dims", [(296, 9, 7), (40, 6, 5), (64, 5, 4)])
@pytest.mark.parametrize("batches", [(1,), (2,), (3, 4)])
def test_bulk_periodic_box(storage, dims, batches):
    """Every face periodic (wrapped rows); nx = 296: one full 256-node tile and an 8-node tail per
    row; nx = 40: one 8-node tile; nx = 64: one 32-node tile."""
    faces = ("periodic",) * 6
    _same(_run(True, dims, faces, storage, batches, u0=(0.03, -0.01, 0.02), rho_noise=0.01),
          _run(False, dims, faces, storage, batches, u0=(0.03, -0.01, 0.02), rho_noise=0.01))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("lateral", [("noslip",) * 4, ("noslip", "noslip", "periodic", "periodic")])
def test_bulk_channel_faces(storage, lateral):
    """Inlet / outlet channel with bounced (no-slip) and wrapped face rows."""
    faces = ("inlet", "outlet") + lateral
    _same(_run(True, (136, 12, 10), faces, storage, (7,), rho_noise=0.005),
          _run(False, (136, 12, 10), faces, storage, (7,), rho_noise=0.005))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_bulk_city_with_solid_and_freeslip(storage):
    """Buildings with the immersed boundary under a free-slip top: the face rows run in the
    free-slip kernels and the bulk kernel takes the rows off the faces, with band forces."""
    dims = (136, 40, 48)
    X, A = scenes.box_city(*dims, n_boxes=10, side_range=(3, 7), height_range=(5, 28), seed=77)
    solid = (X.astype(np.float32), A.astype(np.float32))
    _same(_run(True, dims, CITY_FACES, storage, (2, 3), solid=solid),
          _run(False, dims, CITY_FACES, storage, (2, 3), solid=solid))


def test_bulk_with_tracers():
    """The velocity output of the step (smoke tracers present) from the bulk kernel."""
    dims = (136, 40, 48)
    X, A = scenes.box_city(*dims, n_boxes=10, side_range=(3, 7), height_range=(5, 28), seed=77)
    solid = (X.astype(np.float32), A.astype(np.float32))
    a = _run(True, dims, CITY_FACES, "f16", (4,), solid=solid, tracers=True)
    b = _run(False, dims, CITY_FACES, "f16", (4,), solid=solid, tracers=True)
    _same(a, b)
    assert np.array_equal(a.tracers(), b.tracers())


def test_bulk_wait_flag_clear():
    """The bounded waits of the tensor-copy kernel did not run out: lbm_check and lbm_synchronize pass."""
    s = _run(True, (296, 9, 7), ("periodic",) * 6, "f16", (5,))
    s.synchronize(30.0)
    from paper_2101_11856_gb300 import lbm
    assert lbm.lbm_check(s.h) == lbm.LBM_OK


def test_bulk_wait_limit_expires():
    """The bounded wait of the tensor-copy kernel runs out (self-test mode: every barrier waits for
    16 bytes no copy delivers): LBM_ETIMEOUT reaches the host, the kernel ends by itself, and the
    context keeps working once a state is set again."""
    from paper_2101_11856_gb300 import lbm
    dims = (64, 6, 5)
    s = _run(True, dims, ("periodic",) * 6, "f16", ())
    s.set_pair_kernel(2)
    s.step(1)
    with pytest.raises(lbm.LBMError) as e:
        s.synchronize(60.0)
    assert e.value.code == lbm.LBM_ETIMEOUT
    assert lbm.lbm_check(s.h) == lbm.LBM_OK   # the flag was reported once and cleared
    s.set_pair_kernel(1)
    rho, u = scenes.uniform_flow(*dims, (0.04, 0.0, 0.0))
    s.set_state(rho, u)
    s.step(3)
    s.synchronize(60.0)
    ref = _run(False, dims, ("periodic",) * 6, "f16", (3,))
    _same(s, ref)
