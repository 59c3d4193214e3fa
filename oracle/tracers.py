"""Smoke tracers: advection in the lattice velocity and projection of their density onto a
volume grid (Sec. 6, the paragraph on rendering: smoke particles are traced in parallel on
the GPU and their densities projected onto a uniform volume grid).

ORACLE -- test infrastructure only.

The paper gives no formulas for either step.  Readings used here (and by the library):

* Velocity at a point (lattice units, node k at coordinate k): trilinear interpolation of
  the Guo-shifted velocity u of the last collision (the field ``lbm_macroscopic`` returns).
  Along a periodic axis of n nodes the corners are taken modulo n; along a non-periodic
  axis the base node is min(floor(x), n - 2) (so x = n - 1 uses the last cell with
  weight 1 on its upper node).
* Tracing over one time step (dt = 1): explicit midpoint rule,
  x_mid = x + u(x) / 2, x' = x + u(x_mid).  After each of the two stages the periodic
  coordinates are wrapped into [0, n) (x < 0: x += n, then x >= n: x -= n).
* A tracer whose midpoint or end point leaves [0, n - 1] along a non-periodic axis is
  re-injected (the scenes inject smoke continuously): its new position is lo + (hi - lo) U
  with U_a in [0, 1) the top 24 bits of SplitMix64 (the generator of ``noise``) at counter
  ((t - 1) P + i) 3 + a, times 2^-24, t the 1-based step, P the tracer count, i its index,
  and [lo, hi) the emitter box.
* Density: every tracer carries unit mass, spread by the same trilinear weights
  (cloud-in-cell) onto a grid of spacing s (an integer >= 1, voxel j at coordinate j s).
  A periodic axis has n / s voxels (n divisible by s) and wraps; a non-periodic axis has
  ceil((n - 1) / s) + 1 voxels and base voxel min(floor(x / s), g - 2).
  The sum is a plain scatter-add in FP64 here; the library sorts the contributions by
  voxel and reduces each run (no float atomics), which gives the same sums up to rounding.
"""
from __future__ import annotations

import numpy as np

from .noise import splitmix64


def _axis_stencil(x: np.ndarray, n: int, periodic: bool):
    """Lower/upper node indices and the weight of the upper node along one axis."""
    if periodic:
        b = np.floor(x)
        w = x - b
        lo = np.mod(b.astype(np.int64), n)
        return lo, np.mod(lo + 1, n), w
    b = np.minimum(np.floor(x), n - 2)
    return b.astype(np.int64), b.astype(np.int64) + 1, x - b


def interpolate(u: np.ndarray, X: np.ndarray, periodic) -> np.ndarray:
    """Trilinear interpolation of the field u (3, nz, ny, nx) at points X (P, 3) -> (P, 3)."""
    _, nz, ny, nx = u.shape
    ix0, ix1, wx = _axis_stencil(X[:, 0], nx, periodic[0])
    iy0, iy1, wy = _axis_stencil(X[:, 1], ny, periodic[1])
    iz0, iz1, wz = _axis_stencil(X[:, 2], nz, periodic[2])
    out = np.zeros((X.shape[0], 3))
    for iz, fz in ((iz0, 1.0 - wz), (iz1, wz)):
        for iy, fy in ((iy0, 1.0 - wy), (iy1, wy)):
            for ix, fx in ((ix0, 1.0 - wx), (ix1, wx)):
                out += (fx * fy * fz)[:, None] * u[:, iz, iy, ix].T
    return out


def wrap(X: np.ndarray, shape_xyz, periodic) -> np.ndarray:
    """Periodic coordinates into [0, n): add n if negative, then subtract n if >= n."""
    X = X.copy()
    for a in range(3):
        if periodic[a]:
            n = shape_xyz[a]
            X[:, a] = np.where(X[:, a] < 0.0, X[:, a] + n, X[:, a])
            X[:, a] = np.where(X[:, a] >= n, X[:, a] - n, X[:, a])
    return X


def inside(X: np.ndarray, shape_xyz, periodic) -> np.ndarray:
    """True where every non-periodic coordinate lies in [0, n - 1]."""
    ok = np.ones(X.shape[0], dtype=bool)
    for a in range(3):
        if not periodic[a]:
            ok &= (X[:, a] >= 0.0) & (X[:, a] <= shape_xyz[a] - 1)
    return ok


def emitter_positions(lo, hi, seed: int, t: int, count: int, idx: np.ndarray) -> np.ndarray:
    """Re-injection positions of the tracers ``idx`` at step t (see the module docstring)."""
    out = np.empty((idx.shape[0], 3))
    for a in range(3):
        with np.errstate(over="ignore"):
            ctr = (np.uint64(t - 1) * np.uint64(count) + idx.astype(np.uint64)) * np.uint64(3) + np.uint64(a)
        U = (splitmix64(seed, ctr) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
        out[:, a] = lo[a] + (hi[a] - lo[a]) * U
    return out


def advect(u: np.ndarray, X: np.ndarray, t: int, periodic, emitter) -> np.ndarray:
    """One step of the explicit midpoint rule with re-injection; u (3, nz, ny, nx), X (P, 3).
    ``emitter`` = (lo, hi, seed)."""
    shape_xyz = (u.shape[3], u.shape[2], u.shape[1])
    Xm = wrap(X + 0.5 * interpolate(u, X, periodic), shape_xyz, periodic)
    ok = inside(Xm, shape_xyz, periodic)
    Xn = X.copy()
    if ok.any():
        Xn[ok] = wrap(X[ok] + interpolate(u, Xm[ok], periodic), shape_xyz, periodic)
    ok &= inside(Xn, shape_xyz, periodic)
    bad = np.nonzero(~ok)[0]
    if bad.size:
        lo, hi, seed = emitter
        Xn[bad] = emitter_positions(lo, hi, seed, t, X.shape[0], bad)
    return Xn


def grid_dims(shape_xyz, periodic, s: int):
    """Voxels per axis of the density grid of spacing s."""
    dims = []
    for a in range(3):
        n = shape_xyz[a]
        if periodic[a]:
            assert n % s == 0
            dims.append(n // s)
        else:
            dims.append(-(-(n - 1) // s) + 1)
    return tuple(dims)


def density(X: np.ndarray, shape_xyz, periodic, s: int) -> np.ndarray:
    """Cloud-in-cell density of unit-mass tracers on the grid of spacing s -> (gz, gy, gx)."""
    gx, gy, gz = grid_dims(shape_xyz, periodic, s)
    rho = np.zeros((gz, gy, gx))
    Y = X / s
    ix0, ix1, wx = _axis_stencil(Y[:, 0], gx, periodic[0])
    iy0, iy1, wy = _axis_stencil(Y[:, 1], gy, periodic[1])
    iz0, iz1, wz = _axis_stencil(Y[:, 2], gz, periodic[2])
    for iz, fz in ((iz0, 1.0 - wz), (iz1, wz)):
        for iy, fy in ((iy0, 1.0 - wy), (iy1, wy)):
            for ix, fx in ((ix0, 1.0 - wx), (ix1, wx)):
                np.add.at(rho, (iz, iy, ix), fx * fy * fz)
    return rho
