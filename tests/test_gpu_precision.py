"""FP16 / BF16 deviation storage through the main and edge kernels (nx >= 33), for the three
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


CHANNEL = ("inlet", "outlet", "noslip", "noslip", "periodic", "periodic")
CASES = [(s, c, (70, 6, 5), CHANNEL) for s in ("f16", "bf16", "f32") for c in ("acm", "bgk", "raw")]
# 16-bit storage with the method's collision runs the main range in node pairs when nx is even:
# 68 pairs in two blocks (ragged), no-slip y rows and wrapped z rows; with a free-slip top the
# pair kernel runs the rows off the y/z faces only; nx odd runs one node per thread
CASES += [(s, "acm", dims, CHANNEL) for s in ("f16", "bf16") for dims in ((200, 5, 6), (201, 5, 6))]
CASES += [("f16", "acm", (200, 5, 6), ("inlet", "outlet", "noslip", "freeslip", "periodic", "periodic"))]


@pytest.mark.parametrize("storage,collision,dims,faces", CASES)
def test_one_step_from_stored_state(storage, collision, dims, faces):
    nx, ny, nz = dims
    rho, u = scenes.taylor_green(nx, ny, nz, 0.04)
    u[0] += 0.04
    X, A = scenes.fibonacci_sphere((36.2, ny / 2 - 0.3, nz / 2 - 0.6), 1.6, 30)
    if nx > 100:
        X2, A2 = scenes.fibonacci_sphere((150.7, ny / 2 - 0.2, nz / 2 + 0.1), 1.2, 24)
        X, A = np.concatenate([X, X2]), np.concatenate([A, A2])
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
