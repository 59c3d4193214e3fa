"""One time step of the IB kinetic solver in the paper's order (Algorithm 2, Eqs. 1-8).

ORACLE -- test infrastructure only.

Per step t (1-based), starting from the post-collision populations f(t-1):

1. streaming with the domain faces (Eq. 3; ``streaming``), giving f*;
2. macroscopic moments rho* = sum f*, j = sum c f* (Eq. 2, Algorithm 2 (b));
3. immersed boundary (Algorithm 2 (c)): the velocity seen by the solid is the pre-IB
   velocity u_IB = (j + F_body/2)/rho*; it is interpolated to the samples together with
   rho* (Eq. 6), the penalty force g_s = rho_s (u_b - u_s) dA_s (Eq. 7) is spread to the
   nodes (Eq. 8), and the drag on the solid is -sum_s g_s;
4. collision with the total force F = F_body + F_IB (Eqs. 4-5; ``collision``).

``ib_lag`` (a reading for the fused variant of the step, not the paper's order): step 3 takes
rho* and u_IB from the streamed populations of the previous step instead of this one's (this
one's for the first step after set_state or set_solids); everything else is unchanged.

The macroscopic fields reported for step t are rho* and the Guo-shifted velocity
(j + F/2)/rho* used by that collision; before the first step they are the initial fields.
The initial populations are the equilibrium of the initial fields, taken as the
post-collision state at t = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import collision as col
from . import ib
from . import motion as mo
from .lattice import DTYPE
from .noise import inlet_noise
from .streaming import check_faces, stream


@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    nu: float
    forcing: tuple = (0.0, 0.0, 0.0)
    faces: tuple = ("periodic",) * 6
    rho0: float = 1.0
    u_in: float = 0.0
    noise: float = 0.0
    seed: int = 0
    omega_bulk: float = 1.0
    omega_hi: tuple = (1.0, 1.0, 1.0, 1.0)
    collision: str = "factorised"          # or "matrix" (same operator), "bgk", "raw" (comparison models)
    ib_lag: bool = False                   # step-lagged immersed boundary (see the module docstring)
    rates: dict = field(init=False)

    def __post_init__(self):
        check_faces(self.faces)
        self.rates = col.relaxation_rates(self.nu, self.omega_bulk, self.omega_hi)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def inflow_modes(ny: int, nz: int) -> torch.Tensor:
    """sin(m pi (y+1/2)/ny) sin(n pi (z+1/2)/nz), m, n = 1..4 -> (16, nz, ny), row-major in m."""
    y = (torch.arange(ny, dtype=DTYPE) + 0.5) / ny
    z = (torch.arange(nz, dtype=DTYPE) + 0.5) / nz
    modes = []
    for m in range(1, 5):
        for n in range(1, 5):
            modes.append(torch.sin(n * math.pi * z)[:, None] * torch.sin(m * math.pi * y)[None, :])
    return torch.stack(modes)


def inlet_velocity(p: Problem, t: int, coef: torch.Tensor | None) -> torch.Tensor:
    """u_in(y, z, t) = u_in (1 + noise xi(t, y, z)) + sum_mn a_mn sin(..) sin(..); (nz, ny)."""
    ux = torch.full((p.nz, p.ny), p.u_in, dtype=DTYPE)
    if p.noise != 0.0:
        xi = torch.from_numpy(inlet_noise(p.seed, t, p.ny, p.nz))
        ux = ux * (1.0 + p.noise * xi)
    if coef is not None:
        ux = ux + torch.einsum("k,kzy->zy", coef, inflow_modes(p.ny, p.nz))
    return ux


def collide(p: Problem, fstar, F):
    if p.collision == "matrix":
        return col.collide_matrix(fstar, F, p.rates)
    if p.collision == "bgk":
        return col.collide_bgk(fstar, F, p.rates["shear"])
    if p.collision == "raw":
        return col.collide_raw(fstar, F, p.rates)
    return col.collide_factorised(fstar, F, p.rates)


def step(p: Problem, f: torch.Tensor, t: int, coef=None, solids=None, ib_moments=None):
    """Advance post-collision f(t-1) to f(t).  ``solids`` = (X (S,3), area (S,), u_b (3,S)).
    ``ib_moments`` = (rho*, u_IB) the immersed boundary interpolates instead of this step's
    (the step-lagged variant), or None.

    Returns (f(t), diagnostics dict with rho, u, F, g, drag and this step's rho*, u_IB).
    """
    wall = inlet_velocity(p, t, coef) if "inlet" in p.faces else None
    fstar = stream(f, p.faces, wall, p.rho0)
    rho, j = col.density_momentum(fstar)
    F = torch.tensor(p.forcing, dtype=DTYPE).view(3, 1, 1, 1).expand(3, *p.shape)
    u_ib = col.guo_velocity(rho, j, F)
    g = None
    drag = torch.zeros(3, dtype=DTYPE)
    if solids is not None:
        X, area, u_b = solids
        rho_i, u_i = (rho, u_ib) if ib_moments is None else ib_moments
        rho_s = ib.interpolate(rho_i, X)
        u_s = ib.interpolate(u_i, X)
        g = ib.penalty_force(rho_s, u_s, u_b, area)
        F = F + ib.spread_scatter(g, X, p.shape)
        drag = -g.sum(1)
    fnew = collide(p, fstar, F)
    u = col.guo_velocity(rho, j, F)
    return fnew, dict(rho=rho, u=u, F=F, g=g, drag=drag, u_ib=u_ib)


class OracleSolver:
    """Stateful wrapper with the same operations as the C-ABI library."""

    def __init__(self, p: Problem, inflow_coef=None):
        self.p = p
        self.coef = None if inflow_coef is None else torch.as_tensor(np.asarray(inflow_coef), dtype=DTYPE)
        self.solids = None
        self.motion = None
        self.X0 = None
        self.t = 0
        self.f = None
        self.diag = None
        self.ib_moments = None                # (rho*, u_IB) of the last step's streamed populations

    def set_state(self, rho, u):
        rho = torch.as_tensor(np.asarray(rho), dtype=DTYPE)
        u = torch.as_tensor(np.asarray(u), dtype=DTYPE)
        self.f = col.equilibrium(rho, u)
        self.t = 0
        self.diag = dict(rho=rho.clone(), u=u.clone(), drag=torch.zeros(3, dtype=DTYPE), g=None)
        self.ib_moments = None

    def set_solids(self, X, area=None, u_b=None):
        X = torch.as_tensor(np.asarray(X), dtype=DTYPE)
        S = X.shape[0]
        area = torch.ones(S, dtype=DTYPE) if area is None else torch.as_tensor(np.asarray(area), dtype=DTYPE)
        u_b = torch.zeros(3, S, dtype=DTYPE) if u_b is None else torch.as_tensor(np.asarray(u_b), dtype=DTYPE).T
        self.solids = (X, area, u_b)
        self.motion = None
        self.ib_moments = None

    def set_motion(self, motion):
        """Prescribed rigid motion (c0, V, axis, w) of the current samples (``motion``)."""
        self.motion = motion
        self.X0 = self.solids[0].numpy().copy()
        self.t0 = self.t                      # the samples now are the pose of time 0
        self._pose(self.t)

    def _pose(self, t_abs):
        tau = t_abs - self.t0
        X = mo.sample_positions(self.X0, self.motion, tau)
        ub = mo.boundary_velocity(X, self.motion, tau)
        self.solids = (torch.from_numpy(X), self.solids[1], torch.from_numpy(ub.T.copy()))

    def step(self, n: int = 1):
        for _ in range(n):
            self.t += 1
            if self.motion is not None:
                self._pose(self.t - 1)        # Algorithm 2 (c): the update after the previous IB stage
            lagged = self.ib_moments if self.p.ib_lag else None
            self.f, self.diag = step(self.p, self.f, self.t, self.coef, self.solids, lagged)
            self.ib_moments = (self.diag["rho"], self.diag["u_ib"])

    def torque(self, center):
        """Torque on the solid about ``center`` from the last step's samples and forces."""
        return mo.torque(self.solids[0].numpy(), self.diag["g"].numpy().T, center)

    def macroscopic(self):
        return self.diag["rho"], self.diag["u"]

    def reductions(self):
        rho, u = self.diag["rho"], self.diag["u"]
        mass = float(rho.sum())
        mom = (rho * u).sum((1, 2, 3))
        return mass, mom, self.diag["drag"]

    def populations(self):
        """Post-collision populations of the current time, (27, nz, ny, nx) in lattice order."""
        return self.f
