"""Full-grid parity of the sphere channel 256 x 128 x 128 after 100 steps (the configuration of
the paper's sphere/obstacle channel scenes, Table 3, at the sizes of this workload): Fibonacci
sphere of radius 16 with 3,200 samples, inlet u = 0.05 with 1 % seeded noise, outlet, periodic
y and z, nu = 0.008 (Re = 200), from the uniform inflow state.

The expected density and Guo-shifted velocity (Eq. 2) of the FP64 oracle at about 110,000 cells
(every band node, the inlet and outlet planes, the planes through and behind the sphere and
20,000 seeded cells) are stored in tests/golden/sphere_channel_256x128x128_100steps.npz,
written by tests/golden/make_sphere_channel_golden.py from the oracle alone.

FP32 storage must meet the stated bar, relative L2 <= 1e-5 on rho and on u over the stored
cells, plus absolute bounds.  FP16 and BF16 deviation storage have no pass bar beyond
stability: their error against the oracle is reported per field (rho - 1, u_x, u_y, u_z).
"""
import json
import os

import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "sphere_channel_256x128x128_100steps.npz")


def golden():
    z = np.load(GOLDEN)
    return z["idx"].astype(np.int64), z["rho"], z["u"], json.loads(str(z["meta"]))


def run_gpu(storage, meta):
    from paper_2101_11856_gb300 import Solver, lbm
    s = scenes.scene_sphere_channel(256, 128, 128, radius=meta["radius"], count=meta["count"], u_in=meta["u_in"],
                                    nu=meta["nu"], noise=meta["noise"])
    nx, ny, nz = s["nx"], s["ny"], s["nz"]
    g = Solver(nx, ny, nz, s["nu"], storage=storage, faces=s["faces"], u_in=s["u_in"], noise=s["noise"],
               seed=meta["seed"])
    g.set_state(s["rho"], s["u"])
    g.set_solids(s["samples"].astype(np.float32), s["area"].astype(np.float32))
    g.step(meta["steps"])
    N = nx * ny * nz
    rho = torch.empty(N, device="cuda")
    u = torch.empty(3, N, device="cuda")
    lbm.lbm_macroscopic(g.h, rho, u)
    assert lbm.lbm_check(g.h) == lbm.LBM_OK
    _, _, drag = g.reductions()
    g.close()
    return rho, u, drag


def field_errors(rho_g, u_g, rho_o, u_o):
    """Relative L2 over the stored cells of rho, rho - 1, u (all components) and each component."""
    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"rho": rel(rho_g, rho_o), "rho-1": rel(rho_g - 1.0, rho_o - 1.0), "u": rel(u_g, u_o),
            "u_x": rel(u_g[0], u_o[0]), "u_y": rel(u_g[1], u_o[1]), "u_z": rel(u_g[2], u_o[2])}


@pytest.fixture(scope="module")
def expected():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return golden()


def test_sphere_channel_fp32_100_steps(expected):
    idx, rho_o, u_o, meta = expected
    assert meta["steps"] == 100 and idx.size >= 100_000
    rho, u, drag = run_gpu("f32", meta)
    ti = torch.from_numpy(idx).cuda()
    rho_g = rho[ti].double().cpu().numpy()
    u_g = u[:, ti].double().cpu().numpy()
    e = field_errors(rho_g, u_g, rho_o, u_o)
    du, dr = float(np.abs(u_g - u_o).max()), float(np.abs(rho_g - rho_o).max())
    ddrag = abs(float(drag[0]) - meta["drag"][0]) / abs(meta["drag"][0])
    print("f32 sphere channel 256x128x128, 100 steps, " + ", ".join(f"{k} {v:.2e}" for k, v in e.items())
          + f"; max |du| {du:.2e}, max |drho| {dr:.2e}, drag_x rel {ddrag:.2e}")
    assert e["rho"] <= 1e-5 and e["u"] <= 1e-5
    # absolute: 2e-5 of the inflow speed, and 16 FP32 ulps of 1 in the density
    assert du <= 1e-6 and dr <= 1e-6
    assert ddrag <= 1e-4


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_sphere_channel_reduced_precision_reported(expected, storage):
    idx, rho_o, u_o, meta = expected
    rho, u, drag = run_gpu(storage, meta)
    ti = torch.from_numpy(idx).cuda()
    rho_g = rho[ti].double().cpu().numpy()
    u_g = u[:, ti].double().cpu().numpy()
    e = field_errors(rho_g, u_g, rho_o, u_o)
    print(f"{storage} sphere channel 256x128x128, 100 steps, per field vs the FP64 oracle: "
          + ", ".join(f"{k} {v:.2e}" for k, v in e.items())
          + f"; drag_x {float(drag[0]):.4e} (oracle {meta['drag'][0]:.4e})")
    assert all(np.isfinite(v) for v in e.values())
    assert e["u"] <= 0.05          # stability (BF16 keeps 8 bits of each deviation)
