"""lbm_sum_forces_static: the allocation-free FP64 force sum, for callers that cannot call
cudaMalloc where they need the result.  It must agree with the drag that the
context-based lbm_reductions returns (drag = -sum of the per-sample forces), on two calls
in a row that share its fixed device scratch.  Collected last on purpose."""
import numpy as np
import pytest
import torch

import scenes
from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def test_static_force_sum_matches_reductions_twice():
    need_gpu()
    from paper_2101_11856_gb300 import Solver, lbm
    n = 24
    rho, u = scenes.taylor_green(n, n, n, 0.05)
    X, A = scenes.fibonacci_sphere((11.2, 12.4, 10.7), 6.3, 1500)
    s = Solver(n, n, n, 0.02, forcing=(1e-5, 0.0, 0.0))
    s.set_state(rho, u)
    s.set_solids(X, A, np.tile([0.02, 0.0, -0.01], (1500, 1)))
    g = torch.empty(1500, 3, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    for call in range(2):
        s.step(3)
        lbm.lbm_ib_forces(s.h, g)
        out.fill_(float("nan"))
        lbm.lbm_sum_forces_static(g, out)
        torch.cuda.synchronize()
        _, _, drag = s.reductions()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.abs(got + drag).max() <= 1e-12 * np.abs(drag).max() + 1e-15, (call, got, drag)
    # an empty input gives zeros, and oversized or missing arguments are rejected
    lbm.lbm_sum_forces_static(torch.empty(0, 3, device="cuda"), out)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0.0)
    lib = lbm.library()
    assert lib.lbm_sum_forces_static(None, 5, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_sum_forces_static(g.data_ptr(), 2048 * 256 * 64 + 1, out.data_ptr(), None) == lbm.LBM_EINVAL
    s.close()
