"""Direct-forcing immersed boundary: interpolation, penalty force, spreading (Eqs. 6-8).

ORACLE -- test infrastructure only.

* Kernel (Sec. 3.1, "the smallest 2x2x2 kernel"): the separable trilinear hat
  K(r) = prod_a max(0, 1 - |r_a|); the paper's K(||x_s - x_f||) notation is read as
  this separable kernel.  A sample X has base node b = floor(X) and weight
  prod_a (d_a ? w_a : 1 - w_a), w = X - b, on the 8 nodes b + d, d in {0,1}^3.
* Interpolation (Eq. 6): u(X_s) = sum K u(x_f), and the density likewise.
* Penalty force (Eq. 7): g_s = rho_s (u_b - u_s), multiplied by the sample's area
  weight dA_s (lattice units; the paper does not print one, but with 10-100 samples per
  cell an unweighted sum would scale the force with the sampling density).
* Spreading (Eq. 8): F(x_f) = sum_s K(X_s - x_f) g_s, computed by scatter over samples
  (the paper's load-balanced form, Sec. 4.3.2) and, for small cases, by brute-force
  gather over all samples for every node (the form Eq. 8 is written in).  The paper
  states the two are equivalent; ``tests/test_oracle_ib.py`` checks it.
"""
from __future__ import annotations

import torch

from .lattice import DTYPE

CORNERS = [(dx, dy, dz) for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]


def stencil(X: torch.Tensor):
    """Base nodes (S, 3) int64 and trilinear weights (S, 8) of samples X (S, 3)."""
    b = torch.floor(X)
    w = X - b
    K = torch.stack([
        (w[:, 0] if d[0] else 1.0 - w[:, 0]) * (w[:, 1] if d[1] else 1.0 - w[:, 1])
        * (w[:, 2] if d[2] else 1.0 - w[:, 2]) for d in CORNERS], dim=1)
    return b.to(torch.int64), K


def _flat(b: torch.Tensor, d, shape):
    nz, ny, nx = shape
    return ((b[:, 2] + d[2]) * ny + (b[:, 1] + d[1])) * nx + (b[:, 0] + d[0])


def interpolate(field: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """Eq. 6: field (..., nz, ny, nx) sampled at X (S, 3) -> (..., S)."""
    shape = field.shape[-3:]
    flat = field.reshape(*field.shape[:-3], -1)
    b, K = stencil(X)
    out = 0.0
    for k, d in enumerate(CORNERS):
        out = out + K[:, k] * flat[..., _flat(b, d, shape)]
    return out


def penalty_force(rho_s, u_s, u_b, area) -> torch.Tensor:
    """Eq. 7 with the area weight: g_s = rho_s (u_b - u_s) dA_s, shape (3, S)."""
    return rho_s * (u_b - u_s) * area


def spread_scatter(g: torch.Tensor, X: torch.Tensor, shape) -> torch.Tensor:
    """Eq. 8 by scatter: every sample adds K g to its 8 nodes. g (3, S) -> F (3, nz, ny, nx)."""
    nz, ny, nx = shape
    b, K = stencil(X)
    F = torch.zeros(3, nz * ny * nx, dtype=DTYPE)
    for k, d in enumerate(CORNERS):
        F = F.index_add(1, _flat(b, d, shape), K[:, k] * g)
    return F.reshape(3, nz, ny, nx)


def hat(r: torch.Tensor) -> torch.Tensor:
    """Separable 2x2x2 hat kernel K(r) = prod_a max(0, 1 - |r_a|); r (..., 3)."""
    return torch.clamp(1.0 - r.abs(), min=0.0).prod(-1)


def spread_gather(g: torch.Tensor, X: torch.Tensor, shape) -> torch.Tensor:
    """Eq. 8 as written: for every node sum K(X_s - x_f) g_s over all samples (small cases)."""
    nz, ny, nx = shape
    zz, yy, xx = torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx), indexing="ij")
    nodes = torch.stack([xx, yy, zz], -1).reshape(-1, 3).to(DTYPE)     # (N, 3)
    K = hat(X[None, :, :] - nodes[:, None, :])                           # (N, S)
    return (K @ g.T).T.reshape(3, nz, ny, nx)
