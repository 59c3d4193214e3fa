"""Asynchronous host transfers (lbm_set_state_async, lbm_macroscopic_async): batches of steps
with the uploads and read-backs queued on the copy streams, overlapping the steps, give the
same fields bit for bit as the blocking calls.  Three batches use both input staging buffers
and reuse the first; pinned, pageable and device buffers."""
import numpy as np
import pytest
import torch

import scenes
from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu

DIMS = (80, 12, 10)
BATCHES, STEPS = 3, 7


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def solver():
    from paper_2101_11856_gb300 import Solver
    nx, ny, nz = DIMS
    s = Solver(nx, ny, nz, 0.02, faces=("inlet", "outlet", "noslip", "freeslip", "periodic", "periodic"),
               u_in=0.04, noise=0.01, seed=3)
    X, A = scenes.fibonacci_sphere((40.3, 6.2, 5.1), 2.5, 60)
    s.set_solids(X, A)
    return s


def batch_inputs():
    nx, ny, nz = DIMS
    rng = np.random.default_rng(11)
    out = []
    for b in range(BATCHES):
        rho, u = scenes.uniform_flow(nx, ny, nz, (0.04, 0.0, 0.0))
        rho = (rho + 0.01 * b * rng.standard_normal(rho.shape)).astype(np.float32)
        u = (u + 0.005 * b * rng.standard_normal(u.shape)).astype(np.float32)
        out.append((np.ascontiguousarray(rho), np.ascontiguousarray(u)))
    return out


def blocking(inputs):
    s = solver()
    res = []
    for rho, u in inputs:
        s.set_state(rho, u)
        s.step(STEPS)
        res.append(s.macroscopic())
    s.close()
    return res


@pytest.mark.parametrize("memory", ["pinned", "pageable", "device"])
def test_pipelined_batches_match_blocking(memory):
    inputs = batch_inputs()
    ref = blocking(inputs)
    nx, ny, nz = DIMS
    if memory == "pageable":
        ins = inputs
        outs = [(np.empty((nz, ny, nx), np.float32), np.empty((3, nz, ny, nx), np.float32)) for _ in range(BATCHES)]
    else:
        kw = dict(device="cuda") if memory == "device" else dict(pin_memory=True)
        ins = [(torch.from_numpy(r).to(**kw) if memory == "device" else torch.from_numpy(r).pin_memory(),
                torch.from_numpy(u).to(**kw) if memory == "device" else torch.from_numpy(u).pin_memory())
               for r, u in inputs]
        outs = [(torch.empty((nz, ny, nx), **kw), torch.empty((3, nz, ny, nx), **kw)) for _ in range(BATCHES)]
    s = solver()
    s.set_state_async(*ins[0])
    for b in range(BATCHES):
        s.step(STEPS)
        s.macroscopic_async(*outs[b])
        if b + 1 < BATCHES:
            s.set_state_async(*ins[b + 1])
    s.synchronize(60.0)
    s.close()
    for b in range(BATCHES):
        got = [o.cpu().numpy() if hasattr(o, "cpu") else o for o in outs[b]]
        assert np.array_equal(got[0], ref[b][0]), b
        assert np.array_equal(got[1], ref[b][1]), b


def test_one_field_only():
    """rho alone to the host (u = NULL): the copy stream carries only what was asked for."""
    inputs = batch_inputs()
    ref = blocking(inputs[:1])
    nx, ny, nz = DIMS
    s = solver()
    s.set_state_async(*inputs[0])
    s.step(STEPS)
    rho = np.full((nz, ny, nx), np.nan, np.float32)
    s.macroscopic_async(rho, None)
    s.synchronize(60.0)
    s.close()
    assert np.array_equal(rho, ref[0][0])
