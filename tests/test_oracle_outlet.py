"""Pins of the oracle's outlet rule (the zero-gradient ghost layer on the +x face; reading of
the domain faces, Algorithm 1 and Sec. 4.3.3, where the paper bounces back on every face and
leaves the inlet/outlet types unstated).

The rule: the ghost node (nx, y, z) carries the post-collision populations of (nx-1, y, z),
so a population pulled across the +x face is f*_i(nx-1, y, z) = f_post_i(nx-1, y - c_iy, z - c_iz).

Two independent checks:

* Translation invariance.  A state that does not depend on x stays x-invariant under a
  periodic x axis.  With an inlet on -x and the outlet on +x, the inlet's disturbance
  travels one node per step, so after t steps every node with x >= t must equal the
  periodic run exactly: the ghost of an x-invariant state is the periodic image.  The
  fields vary along y and z, so a flipped or missing lateral shift (y + c_y, z + c_z), or a
  wrap to x = 0 (which the inlet has disturbed after the first step), breaks the equality.
* Plane and shift of one population.  A single post-collision value placed at (nx-1, y0, z0)
  for a direction with c_x = -1 must appear after streaming at (nx-1, y0 + c_y, z0 + c_z)
  (through the ghost) and at (nx-2, y0 + c_y, z0 + c_z) (ordinary streaming), and a value at
  (nx-2, y0, z0) must not reach the ghost: this fixes the plane the ghost copies.
"""
import math

import numpy as np
import pytest
import torch

from oracle.lattice import DTYPE, VELOCITIES
from oracle.solver import OracleSolver, Problem
from oracle.streaming import stream


def xinvariant_state(nx, ny, nz, U, A, case):
    """x-invariant fields on a uniform stream U along x (arrays indexed [z, y, x])."""
    z, y, _ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    u[0] = U
    if case == "shear_z":           # u_y = A sin(2 pi z / nz): transverse shear wave
        u[1] = A * np.sin(2 * math.pi * z / nz)
        rho = np.ones((nz, ny, nx))
    else:                           # both lateral axes vary, density too
        u[1] = A * np.sin(2 * math.pi * z / nz)
        u[2] = 0.7 * A * np.cos(2 * math.pi * y / ny + 0.3)
        u[0] += 0.5 * A * np.sin(2 * math.pi * (y / ny + 2 * z / nz))
        rho = 1.0 + 0.01 * np.cos(2 * math.pi * (2 * y / ny - z / nz))
    return rho, u


@pytest.mark.parametrize("case", ["shear_z", "yz_varying"])
def test_outlet_equals_periodic_image_of_xinvariant_state(case):
    nx, ny, nz, U, A, steps = 14, 6, 8, 0.05, 0.02, 6
    rho, u = xinvariant_state(nx, ny, nz, U, A, case)
    kw = dict(nu=0.03, omega_bulk=1.2, omega_hi=(1.1, 1.3, 0.9, 1.05))
    run = {}
    for label, faces in (("open", ("inlet", "outlet", "periodic", "periodic", "periodic", "periodic")),
                         ("periodic", ("periodic",) * 6)):
        s = OracleSolver(Problem(nx, ny, nz, faces=faces, u_in=U, **kw))
        s.set_state(rho, u)
        hist = []
        for _ in range(steps):
            s.step()
            hist.append(s.populations().clone())
        run[label] = hist
    for t in range(1, steps + 1):
        fo, fp = run["open"][t - 1], run["periodic"][t - 1]
        # the periodic run stays x-invariant (translation symmetry)
        assert (fp - fp[..., :1]).abs().max() < 1e-15
        # nodes the inlet has not reached agree exactly, including the outlet plane x = nx-1
        assert (fo[..., t:] - fp[..., t:]).abs().max() < 1e-15, t
        # and the inlet has reached x = 0 (the comparison is not vacuous)
        assert (fo[..., 0] - fp[..., 0]).abs().max() > 1e-6


def test_outlet_ghost_plane_and_lateral_shift():
    nx, ny, nz = 7, 5, 6
    faces = ("inlet", "outlet", "periodic", "periodic", "periodic", "periodic")
    y0, z0 = 2, 3
    for i, c in enumerate(VELOCITIES):
        if c[0] != -1:
            continue
        f = torch.zeros(27, nz, ny, nx, dtype=DTYPE)
        f[i, z0, y0, nx - 1] = 1.0          # on the outlet plane
        f[i, z0, y0, nx - 2] = 100.0        # one plane upstream
        out = stream(f, faces, torch.zeros(nz, ny, dtype=DTYPE))
        yt, zt = (y0 + c[1]) % ny, (z0 + c[2]) % nz
        assert out[i, zt, yt, nx - 1] == 1.0, c          # through the ghost of the outlet plane
        assert out[i, zt, yt, nx - 2] == 1.0, c          # ordinary streaming from x = nx-1
        assert out[i, zt, yt, nx - 3] == 100.0, c        # ordinary streaming from x = nx-2
        # nothing else carries either value: exactly the three landings
        assert float(out[i].sum()) == 102.0, c
