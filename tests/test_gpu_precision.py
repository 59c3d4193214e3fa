"""FP16 / BF16 deviation storage through the main and edge kernels (nx >= 65), for the three
collision models, one step at a time against the FP64 oracle: the oracle starts from the GPU's own stored populations (read
back exactly), so the only difference left is the storage rounding of the step's output,
half an ulp of each deviation h = f - w rho0 (2^-11 |h| for FP16, 2^-8 |h| for BF16), plus the
FP32 arithmetic of the collision (2e-7) and the FP16 subnormal spacing (6e-8)."""
import numpy as np
import pytest
import torch

import scenes
from gpu_helpers import gpu_order, lib_solver, need_gpu
from oracle.lattice import DTYPE, W
from oracle.solver import OracleSolver, Problem

pytestmark = pytest.mark.gpu

REL = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "f32": 0.0}


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("collision", ["acm", "bgk", "raw"])
@pytest.mark.parametrize("storage", ["f16", "bf16", "f32"])
def test_one_step_from_stored_state(storage, collision):
    nx, ny, nz = 70, 6, 5
    faces = ("inlet", "outlet", "noslip", "noslip", "periodic", "periodic")
    rho, u = scenes.taylor_green(nx, ny, nz, 0.04)
    u[0] += 0.04
    X, A = scenes.fibonacci_sphere((36.2, 2.7, 2.4), 1.6, 30)
    kw = dict(nu=0.03, faces=faces, u_in=0.04, noise=0.01, seed=4, forcing=(1e-5, 0.0, -1e-5))
    g = lib_solver(nx=nx, ny=ny, nz=nz, storage=storage, omega_bulk=1.2, omega_hi=(1.1, 0.95, 1.3, 1.05),
                   collision=collision, **kw)
    g.set_state(rho, u)
    g.set_solids(X, A)
    o = OracleSolver(Problem(nx, ny, nz, omega_bulk=1.2, omega_hi=(1.1, 0.95, 1.3, 1.05),
                             collision={"acm": "factorised", "bgk": "bgk", "raw": "raw"}[collision], **kw))
    o.set_state(rho, u)
    o.set_solids(X, A)
    order = gpu_order()
    w = W.view(27, 1, 1, 1).numpy()
    for t in (1, 2, 3):                      # odd, even, odd AA parity
        fg = g.populations().astype(np.float64)
        o.f = torch.from_numpy(np.stack([fg[order[i]] for i in range(27)]))
        o.t = t - 1
        o.step(1)
        g.step(1)
        fo = o.f.numpy()
        fg = g.populations().astype(np.float64)
        fg = np.stack([fg[order[i]] for i in range(27)])
        h = np.abs(fo - w)
        err = np.abs(fg - fo)
        bound = REL[storage] * h + 2e-7 + 6e-8
        worst = float((err / bound).max())
        print(f"{collision} {storage} step {t}: max |df| {err.max():.2e}, worst error / bound {worst:.2f}")
        assert worst <= 1.0
