"""Full-size parity on sampled cells, in the benchmark's launch configuration, for the
configurations at their full sizes: the buildings benchmark (1200 x 250 x 840, ~3.8M immersed
samples), the 512 x 256 x 256 buildings scene (~1.1M samples) and the 256 x 128 x 128 sphere
channel (3,200 samples); inlet, outlet, no-slip ground and free-slip top (buildings) or
periodic y (sphere), periodic z; FP32, AA in place.

Each run takes 1 or 2 steps from an analytic initial field.  After `k` steps a node depends
only on the initial state within 2k cells (streaming reaches 1 cell per step; the
immersed-boundary force at a node reads samples whose stencils reach 1 more cell).  So for
each sampled cell the FP64 oracle is run on an 11^3 window around it -- with the domain's own
face where the window meets a domain face, and an arbitrary (no-slip) cut elsewhere, 5 cells
away -- and its centre is compared with the GPU's value.  Inlet noise is off here (its
counter uses global coordinates; the small-grid tests cover it).
"""
import math

import numpy as np
import pytest
import torch

import scenes
from oracle.solver import OracleSolver, Problem

pytestmark = pytest.mark.gpu

R = 5


def config(name):
    if name == "box_city_1200x250x840":
        d = scenes.scene_box_city(with_state=False)
    elif name == "box_city_512x256x256":
        d = scenes.scene_box_city(512, 256, 256, n_boxes=200, side_range=(3, 7), u_in=0.05, nu=3.5e-5,
                                  with_state=False)
    else:
        d = scenes.scene_sphere_channel(256, 128, 128, radius=16.0, count=3200, u_in=0.05, nu=0.008)
    return d


def init_fields(x, y, z, dims, u_in):
    """Analytic initial fields at global coordinates (arrays broadcast)."""
    nx, ny, nz = dims
    u = np.stack([u_in + 0.02 * np.sin(2 * math.pi * y / ny) * np.cos(2 * math.pi * z / nz),
                  0.01 * np.sin(2 * math.pi * x / 300.0) * np.ones_like(y * z),
                  0.01 * np.cos(2 * math.pi * z / 210.0) * np.ones_like(x * y)])
    rho = 1.0 + 0.001 * np.cos(2 * math.pi * x / 400.0) * np.sin(2 * math.pi * y / ny) * np.ones_like(z)
    return rho, u


def window(c, n, periodic):
    if periodic:
        return np.arange(c - R, c + R + 1) % n, (False, False), R
    lo, hi = max(0, c - R), min(n - 1, c + R)
    return np.arange(lo, hi + 1), (lo == 0, hi == n - 1), c - lo


def oracle_center(cell, d, X, A, steps):
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    faces_d = d["faces"]
    per = [faces_d[2 * a] == "periodic" for a in range(3)]
    x, y, z = cell
    wins = [window(c, n, p) for c, n, p in zip(cell, (nx, ny, nz), per)]
    faces = []
    for a, (_, (at_lo, at_hi), _) in enumerate(wins):
        faces.append(faces_d[2 * a] if at_lo else "noslip")      # the domain's face, or a far cut
        faces.append(faces_d[2 * a + 1] if at_hi else "noslip")
    (xs, _, cxw), (ys, _, cyw), (zs, _, czw) = wins
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    rho, u = init_fields(Xg.astype(float), Y.astype(float), Z.astype(float), (nx, ny, nz), d["u_in"])
    # samples whose 2x2x2 stencil lies inside the window (positions relative to the window)
    origin = np.array([c - cw for c, cw in zip(cell, (cxw, cyw, czw))], dtype=np.float64)
    rel = X - origin
    for a, n in enumerate((nx, ny, nz)):
        if per[a]:
            rel[:, a] %= n
    keep = np.all((rel >= 0) & (rel < np.array([len(xs) - 1, len(ys) - 1, len(zs) - 1])), 1)
    p = Problem(len(xs), len(ys), len(zs), nu=d["nu"], faces=tuple(faces), u_in=d["u_in"])
    o = OracleSolver(p)
    o.set_state(rho, u)
    if keep.any():
        o.set_solids(rel[keep], A[keep])
    o.step(steps)
    r, v = o.macroscopic()
    return float(r[czw, cyw, cxw]), v[:, czw, cyw, cxw].numpy(), int(keep.sum())


def sample_cells(d, X, rng):
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    cells = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny - 1, 17), (nx - 1, 0, nz - 1), (nx // 2, 0, 0),
             (1, 1, 1), (nx - 2, ny // 2, nz // 2), (0, ny // 2, nz // 2), (nx - 1, ny // 2, nz // 2),
             (nx // 2 + 100, ny - 1, nz // 3)]
    for _ in range(12):
        cells.append((int(rng.integers(0, nx)), int(rng.integers(0, ny)), int(rng.integers(0, nz))))
    for s in rng.choice(len(X), 12, replace=False):     # band nodes next to samples
        b = np.floor(X[s]).astype(int)
        cells.append((int(b[0]), int(b[1]), int(b[2])))
    return cells


@pytest.mark.parametrize("steps", [1, 2])
@pytest.mark.parametrize("name", ["box_city_1200x250x840", "box_city_512x256x256", "sphere_channel_256x128x128"])
def test_fullsize_sampled_cells(name, steps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_11856_gb300 import Solver, lbm
    d = config(name)
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    X, A = d["samples"], d["area"]
    Xf = X.astype(np.float32)
    Af = A.astype(np.float32)
    N = nx * ny * nz
    zz, yy, xx = (torch.arange(n, device="cuda", dtype=torch.float64) for n in (nz, ny, nx))
    s = Solver(nx, ny, nz, d["nu"], faces=d["faces"], u_in=d["u_in"], noise=0.0)
    # the same analytic initial field as init_fields, built on the device plane by plane in FP64
    rho = torch.empty(nz, ny, nx, device="cuda")
    u = torch.empty(3, nz, ny, nx, device="cuda")
    for k in range(nz):
        Y, Xg = torch.meshgrid(yy, xx, indexing="ij")
        zk = torch.full_like(Y, float(k))
        rho[k] = (1.0 + 0.001 * torch.cos(2 * math.pi * Xg / 400.0) * torch.sin(2 * math.pi * Y / ny)).float()
        u[0, k] = (d["u_in"] + 0.02 * torch.sin(2 * math.pi * Y / ny) * torch.cos(2 * math.pi * zk / nz)).float()
        u[1, k] = (0.01 * torch.sin(2 * math.pi * Xg / 300.0)).float()
        u[2, k] = (0.01 * torch.cos(2 * math.pi * zk / 210.0)).float()
    s.set_state(rho.view(-1), u.view(3, -1))
    del rho, u
    s.set_solids(Xf, Af)
    s.step(steps)
    rho_g = torch.empty(N, device="cuda")
    u_g = torch.empty(3, N, device="cuda")
    lbm.lbm_macroscopic(s.h, rho_g, u_g)
    assert lbm.lbm_check(s.h) == lbm.LBM_OK
    rng = np.random.default_rng(7)
    worst_u, worst_r, with_ib = 0.0, 0.0, 0
    for (x, y, z) in sample_cells(d, X, rng):
        idx = x + nx * (y + ny * z)
        rg = float(rho_g[idx])
        ug = u_g[:, idx].cpu().numpy().astype(np.float64)
        ro, uo, ns = oracle_center((x, y, z), d, Xf.astype(np.float64), Af.astype(np.float64), steps)
        with_ib += ns > 0
        worst_r = max(worst_r, abs(rg - ro))
        worst_u = max(worst_u, float(np.abs(ug - uo).max()))
    s.close()
    del rho_g, u_g
    torch.cuda.empty_cache()
    print(f"{name}, {steps} step(s): max |d rho| {worst_r:.2e}, max |d u| {worst_u:.2e}, cells near samples {with_ib}")
    assert with_ib >= 10
    assert worst_r <= 2e-6 and worst_u <= 2e-6
