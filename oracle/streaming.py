"""Two-lattice pull streaming with the domain faces (Eq. 3, Algorithm 1, Sec. 4.3.3).

ORACLE -- test infrastructure only.

f*_i(x) = f_i(x - c_i) (Eq. 3).  The paper treats the domain faces after collision with
bounce-back (Algorithm 1; one kernel per face, Algorithm 2 (e)) and does not state the
inlet/outlet rules; the readings below are applied to the post-collision values of the
previous step while they are pulled, which is the same order (collide, faces, stream).

For a population whose source x - c_i lies outside the domain:

* periodic face: the source wraps around;
* ``noslip``: half-way bounce-back, f*_i(x) = f_post_opp(i)(x);
* ``inlet`` (only on -x): moving-wall bounce-back,
  f*_i(x) = f_post_opp(i)(x) + 2 w_i rho0 (c_i . u_w) / c_s^2 with the wall velocity
  u_w = (u_in(y, z, t), 0, 0) and the reference density rho0;
* ``outlet`` (only on +x): zero-gradient ghost layer, the ghost node (nx, y, z) carries
  the post-collision populations of (nx - 1, y, z), so
  f*_i(nx-1, y, z) = f_post_i(nx-1, y - c_iy, z - c_iz) (lateral wrap if periodic);
* ``freeslip`` (only on y and z faces): half-way specular reflection; the population that
  left the tangential neighbour towards the wall comes back mirrored in the wall's normal:
  for each free-slip axis a crossed by x - c_i the source keeps x_a and the direction takes
  -c_ia, f*_i(x) = f_post_i'(x - c_i + c_ia e_a), c_i' = c_i - 2 c_ia e_a.

When a source crosses several faces (edges, corners) no-slip wins over the inlet, both win
over free-slip, and free-slip is applied before the outlet (the outlet ghost is read at the
mirrored source).
"""
from __future__ import annotations

import torch

from .lattice import CS2, OPPOSITE, VELOCITIES, W

FACES = ("-x", "+x", "-y", "+y", "-z", "+z")
FACE_TYPES = ("periodic", "noslip", "inlet", "outlet", "freeslip")


def check_faces(faces) -> None:
    if len(faces) != 6 or any(t not in FACE_TYPES for t in faces):
        raise ValueError(f"bad face types {faces}")
    for a in range(3):
        if (faces[2 * a] == "periodic") != (faces[2 * a + 1] == "periodic"):
            raise ValueError("periodic faces come in pairs")
    for k, t in enumerate(faces):
        if t == "inlet" and k != 0:
            raise ValueError("the inlet is the -x face")
        if t == "outlet" and k != 1:
            raise ValueError("the outlet is the +x face")
        if t == "freeslip" and k < 2:
            raise ValueError("free-slip faces are y or z faces")


def stream(f_post: torch.Tensor, faces, wall_ux=None, rho0: float = 1.0) -> torch.Tensor:
    """Pull-stream post-collision populations f_post (27, nz, ny, nx) -> f* (27, nz, ny, nx).

    ``wall_ux`` (nz, ny) is the inlet wall velocity u_in(y, z, t) for this step.
    """
    check_faces(faces)
    _, nz, ny, nx = f_post.shape
    z = torch.arange(nz).view(nz, 1, 1)
    y = torch.arange(ny).view(1, ny, 1)
    x = torch.arange(nx).view(1, 1, nx)
    coord = (x, y, z)
    size = (nx, ny, nz)
    out = []
    for i, c in enumerate(VELOCITIES):
        # periodic shift: value at x comes from x - c_i (torch.roll: out[k] = in[k - s])
        fs = torch.roll(f_post[i], shifts=(c[2], c[1], c[0]), dims=(0, 1, 2))
        cross = {}
        for a in range(3):
            src = coord[a] - c[a]
            cross[FACES[2 * a]] = (src < 0).expand(nz, ny, nx)
            cross[FACES[2 * a + 1]] = (src > size[a] - 1).expand(nz, ny, nx)
        kinds = {t: torch.zeros(nz, ny, nx, dtype=torch.bool) for t in FACE_TYPES}
        for face, t in zip(FACES, faces):
            kinds[t] = kinds[t] | cross[face]
        noslip = kinds["noslip"]
        inlet = kinds["inlet"] & ~noslip
        outlet = kinds["outlet"] & ~noslip & ~inlet
        # free-slip crossings per axis (y, z), where no-slip and inlet do not win
        fsy = (cross["-y"] & (faces[2] == "freeslip")) | (cross["+y"] & (faces[3] == "freeslip"))
        fsz = (cross["-z"] & (faces[4] == "freeslip")) | (cross["+z"] & (faces[5] == "freeslip"))
        fsy = fsy & ~noslip & ~inlet
        fsz = fsz & ~noslip & ~inlet
        plain = ~fsy & ~fsz
        bounce = f_post[OPPOSITE[i]]
        fs = torch.where(noslip, bounce, fs)
        if bool(inlet.any()):
            corr = 2.0 * W[i] * rho0 * c[0] * wall_ux.view(nz, ny, 1) / CS2
            fs = torch.where(inlet, bounce + corr, fs)
        if bool((outlet & plain).any()):
            ghost = torch.roll(f_post[i][:, :, nx - 1], shifts=(c[2], c[1]), dims=(0, 1))
            fs = torch.where(outlet & plain, ghost.view(nz, ny, 1).expand(nz, ny, nx), fs)
        for my, mz in ((1, 0), (0, 1), (1, 1)):
            sel = (fsy if my else ~fsy) & (fsz if mz else ~fsz)
            if not bool(sel.any()):
                continue
            cm = (c[0], -c[1] if my else c[1], -c[2] if mz else c[2])
            im = VELOCITIES.index(cm)
            sy, sz = (0 if my else c[1]), (0 if mz else c[2])
            val = torch.roll(f_post[im], shifts=(sz, sy, c[0]), dims=(0, 1, 2))
            fs = torch.where(sel & ~outlet, val, fs)
            if bool((sel & outlet).any()):
                ghost = torch.roll(f_post[im][:, :, nx - 1], shifts=(sz, sy), dims=(0, 1))
                fs = torch.where(sel & outlet, ghost.view(nz, ny, 1).expand(nz, ny, nx), fs)
        out.append(fs)
    return torch.stack(out)
