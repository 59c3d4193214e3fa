"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *generates inputs*: initial density/velocity fields, immersed-solid
surface samples with their area weights, and inflow-profile parameters.  It holds no
step of the lattice Boltzmann method itself (no equilibrium, streaming, collision or
immersed-boundary arithmetic), so that the FP64 oracle and the CUDA path can both be
fed from it without sharing any of the method's computation.

The paper's scenes (meshes of an airplane, dragon, car, building reconstruction; see
the paper's Table 3 and Fig. 1) are not available, so procedural stand-ins with the
same grid sizes and sample counts are generated here:

* ``taylor_green``      -- 3D Taylor-Green vortex (periodic cube, no solids).
* ``shear_wave`` / ``taylor_green_2d`` -- exact decaying Navier-Stokes solutions used to
  pin the viscosity of the collision operator.
* ``fibonacci_sphere``  -- a sphere sampled on a Fibonacci lattice (stand-in for the
  paper's Poisson-disk surface sampling of Sec. 3.1).
* ``box_city``          -- procedural "buildings": axis-aligned boxes standing on the
  ground, every exposed face sampled on a regular sub-cell lattice (stand-in for the
  1200x250x840 building scene of Fig. 1 with ~3.7M samples).

All arrays are float64 numpy; fields are indexed ``[z, y, x]`` and vectors carry the
component first (``u[0]`` is u_x).  Node (i, j, k) sits at position (x, y, z) = (i, j, k)
in lattice units.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 2101


def taylor_green(nx: int, ny: int, nz: int, u0: float, rho0: float = 1.0):
    """3D Taylor-Green vortex with its pressure field.

    u =  u0 sin(kx) cos(ky) cos(kz),  v = -u0 cos(kx) sin(ky) cos(kz),  w = 0,
    p = p0 + rho0 u0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2),  rho = rho0 + (p - p0)/c_s^2,
    with k = 2 pi / n along each axis and c_s^2 = 1/3.
    """
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = 2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    u[1] = -u0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z)
    dp = rho0 * u0 * u0 / 16.0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y)) * (np.cos(2 * kz * z) + 2.0)
    rho = rho0 + 3.0 * dp
    return rho, u


def shear_wave(n: int, amplitude: float, rho0: float = 1.0, background=(0.0, 0.0, 0.0)):
    """Transverse shear wave u_x = A sin(2 pi z / n) on an n^3 periodic cube.

    An exact solution of the incompressible Navier-Stokes equations: the amplitude decays
    as exp(-nu k^2 t), k = 2 pi / n.  ``background`` adds a uniform velocity.
    """
    z = np.arange(n)[:, None, None] * np.ones((n, n, n))
    u = np.zeros((3, n, n, n))
    u[0] = amplitude * np.sin(2 * math.pi * z / n)
    for a in range(3):
        u[a] += background[a]
    rho = np.full((n, n, n), rho0)
    return rho, u


def taylor_green_2d(n: int, amplitude: float, nz: int = 4, rho0: float = 1.0):
    """z-invariant Taylor-Green vortex on an n x n x nz periodic box (exact NS solution).

    u = A sin(kx) cos(ky), v = -A cos(kx) sin(ky); velocity decays as exp(-2 nu k^2 t)
    and the pressure is p = p0 + rho0 A^2/4 (cos 2kx + cos 2ky).
    """
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    k = 2 * math.pi / n
    u = np.zeros((3, nz, n, n))
    u[0] = amplitude * np.sin(k * x) * np.cos(k * y)
    u[1] = -amplitude * np.cos(k * x) * np.sin(k * y)
    rho = rho0 + 3.0 * rho0 * amplitude ** 2 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    return rho, u


def uniform_flow(nx: int, ny: int, nz: int, u=(0.0, 0.0, 0.0), rho0: float = 1.0):
    """Uniform density and velocity (initial state of the channel scenes)."""
    vel = np.zeros((3, nz, ny, nx))
    for a in range(3):
        vel[a] = u[a]
    return np.full((nz, ny, nx), rho0), vel


def fibonacci_sphere(center, radius: float, count: int):
    """``count`` points on a sphere from the Fibonacci lattice.

    z_i = 1 - (2i+1)/count, phi_i = i * pi * (3 - sqrt 5); each point carries the
    area weight 4 pi r^2 / count (lattice units).
    """
    i = np.arange(count, dtype=np.float64)
    zz = 1.0 - (2.0 * i + 1.0) / count
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - zz * zz))
    pts = np.stack([rxy * np.cos(phi), rxy * np.sin(phi), zz], axis=1) * radius
    pts += np.asarray(center, dtype=np.float64)[None, :]
    area = np.full(count, 4.0 * math.pi * radius * radius / count)
    return pts, area


def torus(center, R: float, r: float, spacing: float):
    """Samples on a torus of major radius R and minor radius r about the z axis through
    ``center``: a (theta, phi) grid with ~``spacing`` between neighbours on the outer
    equator, each sample weighted by its patch area r (R + r cos phi) dtheta dphi."""
    nt = max(3, int(round(2.0 * math.pi * (R + r) / spacing)))
    nph = max(3, int(round(2.0 * math.pi * r / spacing)))
    th = (np.arange(nt) + 0.5) * 2.0 * math.pi / nt
    ph = (np.arange(nph) + 0.5) * 2.0 * math.pi / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    ring = R + r * np.cos(P)
    pts = np.stack([ring * np.cos(T), ring * np.sin(T), r * np.sin(P)], axis=-1).reshape(-1, 3)
    pts += np.asarray(center, dtype=np.float64)[None, :]
    area = (r * ring * (2.0 * math.pi / nt) * (2.0 * math.pi / nph)).reshape(-1)
    return pts, area


def _face_lattice(u_lo, u_hi, v_lo, v_hi, spacing):
    nu_ = max(1, int(round((u_hi - u_lo) / spacing)))
    nv_ = max(1, int(round((v_hi - v_lo) / spacing)))
    us = u_lo + (np.arange(nu_) + 0.5) * (u_hi - u_lo) / nu_
    vs = v_lo + (np.arange(nv_) + 0.5) * (v_hi - v_lo) / nv_
    uu, vv = np.meshgrid(us, vs, indexing="ij")
    da = (u_hi - u_lo) / nu_ * (v_hi - v_lo) / nv_
    return uu.ravel(), vv.ravel(), da


def box_city(nx: int, ny: int, nz: int, n_boxes: int = 200, side_range=(3, 7),
             height_range=(20, 120), spacing: float = 0.5, seed: int = SEED,
             x_range=(0.2, 0.8)):
    """Procedural 'buildings': ``n_boxes`` axis-aligned boxes standing on the ground (y = 0).

    Footprint sides are integers uniform in ``side_range``, heights uniform in
    ``height_range`` (clipped below the top of the domain), centres uniform in
    x in [x_range[0] nx, x_range[1] nx] and z in the domain.  Overlaps are allowed and
    interior faces are kept.  The four side faces and the roof of each box are sampled
    at cell-centred points of a ``spacing`` lattice; each sample carries the area of its
    patch.  Every sample satisfies 0 <= X < n - 1 on every axis (boxes are clipped to
    [1, n - 2] laterally).  Returns (samples (S, 3) float64, area (S,) float64).
    """
    rng = np.random.default_rng(seed)
    pts, areas = [], []
    for _ in range(n_boxes):
        wx = int(rng.integers(side_range[0], side_range[1] + 1))
        wz = int(rng.integers(side_range[0], side_range[1] + 1))
        h = float(rng.uniform(height_range[0], height_range[1]))
        cx = float(rng.uniform(x_range[0] * nx, x_range[1] * nx))
        cz = float(rng.uniform(0.0, nz))
        x0, x1 = max(1.0, cx - wx / 2), min(nx - 2.0, cx + wx / 2)
        z0, z1 = max(1.0, cz - wz / 2), min(nz - 2.0, cz + wz / 2)
        h = min(h, ny - 2.0)
        if x1 - x0 < spacing or z1 - z0 < spacing:
            continue
        # side faces x = x0 and x = x1 (coordinates y, z)
        for xf in (x0, x1):
            yy, zz, da = _face_lattice(0.0, h, z0, z1, spacing)
            pts.append(np.stack([np.full_like(yy, xf), yy, zz], 1)); areas.append(np.full(yy.size, da))
        # side faces z = z0 and z = z1 (coordinates x, y)
        for zf in (z0, z1):
            xx, yy, da = _face_lattice(x0, x1, 0.0, h, spacing)
            pts.append(np.stack([xx, yy, np.full_like(xx, zf)], 1)); areas.append(np.full(xx.size, da))
        # roof y = h (coordinates x, z)
        xx, zz, da = _face_lattice(x0, x1, z0, z1, spacing)
        pts.append(np.stack([xx, np.full_like(xx, h), zz], 1)); areas.append(np.full(xx.size, da))
    X = np.concatenate(pts, 0)
    A = np.concatenate(areas, 0)
    return X, A


def inflow_coefficients(scale: float = 0.0, seed: int = SEED):
    """16 Fourier coefficients a_mn (m, n = 1..4, row-major in m) of the inflow profile."""
    if scale == 0.0:
        return np.zeros(16)
    return np.random.default_rng(seed).uniform(-scale, scale, 16)


# --- named workloads (grid sizes and sample counts of the synthetic scenes) -----------

def scene_tgv32():
    """3D Taylor-Green vortex, periodic 32^3, u0 = 0.05, nu = 0.01, rho0 = 1, no solids."""
    rho, u = taylor_green(32, 32, 32, 0.05)
    return dict(name="tgv32", nx=32, ny=32, nz=32, nu=0.01, rho=rho, u=u,
                faces=("periodic",) * 6, samples=None, area=None)


def scene_sphere_channel(nx=256, ny=128, nz=128, radius=16.0, count=3200, u_in=0.05, nu=0.008,
                         center=None, noise=0.01):
    """Channel past an immersed sphere: inlet at x = 0, outlet at x = nx-1, y/z periodic."""
    if center is None:
        center = (nx / 4.0, ny / 2.0, nz / 2.0)
    X, A = fibonacci_sphere(center, radius, count)
    rho, u = uniform_flow(nx, ny, nz, (u_in, 0.0, 0.0))
    return dict(name=f"sphere_channel_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, nu=nu, rho=rho, u=u,
                faces=("inlet", "outlet", "periodic", "periodic", "periodic", "periodic"),
                samples=X, area=A, u_in=u_in, noise=noise)


def scene_rotating_torus(nx=400, ny=200, nz=400, R=40.0, r=12.0, spacing=0.68, omega=0.0015, nu=1e-4):
    """A torus tumbling about the x axis in still air (the rotating-torus scene of the
    paper's Table 3: 400 x 200 x 400, about 53k samples): no-slip ground and top, periodic
    x and z; tip speed omega (R + r) = 0.078."""
    c = (nx / 2.0, ny / 2.0, nz / 2.0)
    X, A = torus(c, R, r, spacing)
    rho, u = uniform_flow(nx, ny, nz, (0.0, 0.0, 0.0))
    return dict(name=f"rotating_torus_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, nu=nu, rho=rho, u=u,
                faces=("periodic", "periodic", "noslip", "noslip", "periodic", "periodic"), samples=X, area=A,
                motion=(c, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), omega))


def scene_box_city(nx=1200, ny=250, nz=840, n_boxes=200, side_range=(8, 24), u_in=0.08, nu=1e-4,
                   spacing=0.5, seed=SEED, noise=0.01, with_state=True):
    """Buildings scene: inlet at x = 0, outlet at x = nx-1, no-slip ground (y = 0), free-slip
    top (y = ny-1), z periodic; ``n_boxes`` procedural boxes sampled at ``spacing``."""
    X, A = box_city(nx, ny, nz, n_boxes, side_range, (20, 120), spacing, seed)
    d = dict(name=f"box_city_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, nu=nu,
             faces=("inlet", "outlet", "noslip", "freeslip", "periodic", "periodic"),
             samples=X, area=A, u_in=u_in, noise=noise)
    if with_state:
        d["rho"], d["u"] = uniform_flow(nx, ny, nz, (u_in, 0.0, 0.0))
    return d
