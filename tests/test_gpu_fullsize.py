"""Full-size parity on sampled cells, in the benchmark's launch configuration.

The benchmark workload (1200 x 250 x 840 cells, ~3.8M immersed samples, inlet, outlet,
no-slip ground/top, periodic z; FP32, AA in place) is run on the GPU for 1 and 2 steps
from an analytic initial field.  After `k` steps a node depends only on the initial
state within 2k cells (streaming reaches 1 cell per step; the immersed-boundary force
at a node reads samples whose stencils reach 1 more cell).  So for each sampled cell the
FP64 oracle is run on an 11^3 window around it -- with the domain's own face where the
window meets a domain face, and an arbitrary (no-slip) cut elsewhere, 5 cells away --
and its centre is compared with the GPU's value.  Inlet noise is off here (its counter
uses global coordinates; the small-grid tests cover it).
"""
import math

import numpy as np
import pytest
import torch

import scenes
from oracle.solver import OracleSolver, Problem

pytestmark = pytest.mark.gpu

NX, NY, NZ = 1200, 250, 840
R = 5


def init_fields(x, y, z):
    """Analytic initial fields at global coordinates (arrays broadcast)."""
    u = np.stack([0.08 + 0.02 * np.sin(2 * math.pi * y / NY) * np.cos(2 * math.pi * z / NZ),
                  0.01 * np.sin(2 * math.pi * x / 300.0) * np.ones_like(y * z),
                  0.01 * np.cos(2 * math.pi * z / 210.0) * np.ones_like(x * y)])
    rho = 1.0 + 0.001 * np.cos(2 * math.pi * x / 400.0) * np.sin(2 * math.pi * y / NY) * np.ones_like(z)
    return rho, u


def window(c, n, periodic):
    if periodic:
        return np.arange(c - R, c + R + 1) % n, ("noslip", "noslip"), R
    lo, hi = max(0, c - R), min(n - 1, c + R)
    return np.arange(lo, hi + 1), ("domain_lo" if lo == 0 else "noslip", "domain_hi" if hi == n - 1 else "noslip"), c - lo


def oracle_center(cell, X, A, steps, nu):
    x, y, z = cell
    xs, (xl, xh), cx = window(x, NX, False)
    ys, (yl, yh), cy = window(y, NY, False)
    zs, (zl, zh), cz = window(z, NZ, True)
    faces = ("inlet" if xl == "domain_lo" else "noslip", "outlet" if xh == "domain_hi" else "noslip",
             "noslip", "noslip", zl, zh)
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    rho, u = init_fields(Xg.astype(float), Y.astype(float), Z.astype(float))
    # samples whose 2x2x2 stencil lies inside the window (positions relative to the window)
    rel = np.stack([X[:, 0] - xs[0], X[:, 1] - ys[0], (X[:, 2] - (z - cz)) % NZ], 1)
    keep = np.all((rel >= 0) & (rel < np.array([len(xs) - 1, len(ys) - 1, len(zs) - 1])), 1)
    p = Problem(len(xs), len(ys), len(zs), nu=nu, faces=faces, u_in=0.08)
    o = OracleSolver(p)
    o.set_state(rho, u)
    if keep.any():
        o.set_solids(rel[keep], A[keep])
    o.step(steps)
    r, v = o.macroscopic()
    return float(r[cz, cy, cx]), v[:, cz, cy, cx].numpy(), int(keep.sum())


def sample_cells(X, rng):
    cells = [(0, 0, 0), (NX - 1, NY - 1, NZ - 1), (0, NY - 1, 17), (NX - 1, 0, NZ - 1), (600, 0, 0),
             (1, 1, 1), (NX - 2, 124, 419), (0, 125, 420), (NX - 1, 125, 420), (700, NY - 1, 300)]
    for _ in range(12):
        cells.append((int(rng.integers(0, NX)), int(rng.integers(0, NY)), int(rng.integers(0, NZ))))
    for s in rng.choice(len(X), 12, replace=False):     # band nodes next to samples
        b = np.floor(X[s]).astype(int)
        cells.append((int(b[0]), int(b[1]), int(b[2])))
    return cells


@pytest.mark.parametrize("steps", [1, 2])
def test_fullsize_sampled_cells(steps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_11856_gb300 import Solver, lbm
    d = scenes.scene_box_city(with_state=False)
    X, A = d["samples"], d["area"]
    Xf = X.astype(np.float32)
    Af = A.astype(np.float32)
    N = NX * NY * NZ
    zz, yy, xx = (torch.arange(n, device="cuda", dtype=torch.float64) for n in (NZ, NY, NX))
    s = Solver(NX, NY, NZ, d["nu"], faces=d["faces"], u_in=0.08, noise=0.0)
    # the same analytic initial field as init_fields, built on the device plane by plane in FP64
    rho = torch.empty(NZ, NY, NX, device="cuda")
    u = torch.empty(3, NZ, NY, NX, device="cuda")
    for k in range(NZ):
        Y, Xg = torch.meshgrid(yy, xx, indexing="ij")
        zk = torch.full_like(Y, float(k))
        rho[k] = (1.0 + 0.001 * torch.cos(2 * math.pi * Xg / 400.0) * torch.sin(2 * math.pi * Y / NY)).float()
        u[0, k] = (0.08 + 0.02 * torch.sin(2 * math.pi * Y / NY) * torch.cos(2 * math.pi * zk / NZ)).float()
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
    for (x, y, z) in sample_cells(X, rng):
        idx = x + NX * (y + NY * z)
        rg = float(rho_g[idx])
        ug = u_g[:, idx].cpu().numpy().astype(np.float64)
        ro, uo, ns = oracle_center((x, y, z), Xf.astype(np.float64), Af.astype(np.float64), steps, d["nu"])
        with_ib += ns > 0
        worst_r = max(worst_r, abs(rg - ro))
        worst_u = max(worst_u, float(np.abs(ug - uo).max()))
    s.close()
    print(f"full size, {steps} step(s): max |d rho| {worst_r:.2e}, max |d u| {worst_u:.2e}, cells near samples {with_ib}")
    assert with_ib >= 10
    assert worst_r <= 2e-6 and worst_u <= 2e-6
