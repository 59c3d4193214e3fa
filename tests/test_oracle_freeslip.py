"""Pins of the oracle's free-slip faces (half-way specular reflection) against the mirror
construction: a free-slip wall at y = -1/2 (and ny - 1/2) acts exactly like the periodic
domain of twice the height holding the mirror image of the state, f_i(y') = f_i'(y) with
y' = 2 ny - 1 - y and c_i' the y-mirrored velocity.  With inlet and outlet x faces the
same holds (corners included), and a body force along the wall drives plug flow (no
wall friction) with the exact history u(t) = (t - 1/2) F / rho (no no-slip reading fits).
No GPU."""
import numpy as np
import pytest
import torch

import scenes
from oracle.lattice import DTYPE, VELOCITIES
from oracle.solver import OracleSolver, Problem


def mirrored(field_rho, field_u, axis):
    """Extend (rho, u) by the mirror image along y (axis 1) or z (axis 0) of (nz, ny, nx)."""
    rho_m = torch.flip(field_rho, dims=(axis,))
    u_m = torch.flip(field_u, dims=(axis + 1,)).clone()
    u_m[2 - axis] = -u_m[2 - axis]            # y: component 1 (axis 1), z: component 2 (axis 0)
    return torch.cat([field_rho, rho_m], dim=axis), torch.cat([field_u, u_m], dim=axis + 1)


@pytest.mark.parametrize("xfaces", [("periodic", "periodic"), ("inlet", "outlet")])
@pytest.mark.parametrize("axes", ["y", "z", "yz"])
def test_freeslip_equals_mirrored_periodic(xfaces, axes):
    nx, ny, nz = 9, 4, 3
    rho, u = scenes.taylor_green(nx, ny, nz, 0.05)
    rho = torch.as_tensor(rho, dtype=DTYPE)
    u = torch.as_tensor(u, dtype=DTYPE)
    u[0] += 0.02
    faces = list(xfaces) + ["periodic"] * 4
    rho2, u2, ny2, nz2 = rho, u, ny, nz
    if "y" in axes:
        faces[2] = faces[3] = "freeslip"
        rho2, u2 = mirrored(rho2, u2, 1)
        ny2 *= 2
    if "z" in axes:
        faces[4] = faces[5] = "freeslip"
        rho2, u2 = mirrored(rho2, u2, 0)
        nz2 *= 2
    faces2 = list(xfaces) + ["periodic"] * 4
    kw = dict(nu=0.03, forcing=(2e-5, 0.0, 0.0), omega_bulk=1.2, omega_hi=(1.1, 0.9, 1.3, 1.05), u_in=0.03)
    a = OracleSolver(Problem(nx, ny, nz, faces=tuple(faces), **kw))
    a.set_state(rho, u)
    b = OracleSolver(Problem(nx, ny2, nz2, faces=tuple(faces2), **kw))
    b.set_state(rho2, u2)
    a.step(6)
    b.step(6)
    assert (a.f - b.f[:, :nz, :ny, :]).abs().max() < 1e-13


def test_plug_flow_between_freeslip_walls():
    n = (6, 5, 4)
    rho, u = scenes.uniform_flow(*n, (0.0, 0.0, 0.0))
    F = 3e-5
    o = OracleSolver(Problem(*n, nu=0.05, forcing=(F, 0.0, 0.0),
                             faces=("periodic", "periodic", "freeslip", "freeslip", "freeslip", "freeslip")))
    o.set_state(rho, u)
    for t in range(1, 11):
        o.step(1)
        ux = o.macroscopic()[1][0]
        assert (ux - (t - 0.5) * F).abs().max() < 1e-15
    # between no-slip walls the same force gives a sheared, slower profile
    p = OracleSolver(Problem(*n, nu=0.05, forcing=(F, 0.0, 0.0),
                             faces=("periodic", "periodic", "noslip", "noslip", "freeslip", "freeslip")))
    p.set_state(rho, u)
    p.step(10)
    uy = p.macroscopic()[1][0].mean((0, 2))
    assert float(uy.max() - uy.min()) > 1e-5


def test_freeslip_conserves_mass_and_tangential_momentum():
    n = (7, 6, 5)
    rho, u = scenes.taylor_green(*n, 0.04)
    o = OracleSolver(Problem(*n, nu=0.02, faces=("periodic", "periodic", "freeslip", "freeslip", "periodic", "periodic")))
    o.set_state(rho, u)
    m0 = float(o.f.sum())
    px0 = float((o.f * torch.tensor([c[0] for c in VELOCITIES], dtype=DTYPE).view(27, 1, 1, 1)).sum())
    o.step(8)
    assert abs(float(o.f.sum()) - m0) < 1e-12 * m0
    px = float((o.f * torch.tensor([c[0] for c in VELOCITIES], dtype=DTYPE).view(27, 1, 1, 1)).sum())
    assert abs(px - px0) < 1e-13
