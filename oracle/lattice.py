"""D3Q27 velocity set (Eq. 1 and the lattice-structure figure of Sec. 3).

ORACLE -- test infrastructure only.

The paper uses the D3Q27 lattice, every c_i landing on a neighbouring node, and defers
the ordering of the 27 velocities to its supplement.  The oracle orders them as
0 = rest, 1-6 = faces, 7-18 = edges, 19-26 = corners, with opposite pairs adjacent
(1|2, 3|4, ...).  Weights are the products of the 1-D weights 2/3 (c = 0) and
1/6 (c = +-1), i.e. 8/27, 2/27, 1/54, 1/216.  Lattice units: dx = dt = 1, c_s^2 = 1/3.
"""
from __future__ import annotations

import torch

DTYPE = torch.float64
CS2 = 1.0 / 3.0


def _ordered_velocities():
    vel = [(0, 0, 0)]
    for a in range(3):                      # faces: +e_a, -e_a
        for s in (1, -1):
            v = [0, 0, 0]
            v[a] = s
            vel.append(tuple(v))
    for a, b in ((0, 1), (0, 2), (1, 2)):   # edges, opposite pairs adjacent
        for sa, sb in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
            v = [0, 0, 0]
            v[a], v[b] = sa, sb
            vel.append(tuple(v))
    for s in ((1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1),   # corners
              (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1)):
        vel.append(s)
    return vel


VELOCITIES = _ordered_velocities()
Q = len(VELOCITIES)
C = torch.tensor(VELOCITIES, dtype=torch.int64)          # (27, 3)
CF = C.to(DTYPE)
OPPOSITE = [VELOCITIES.index(tuple(-c for c in v)) for v in VELOCITIES]


def _w1(c: int) -> float:
    return 2.0 / 3.0 if c == 0 else 1.0 / 6.0


W = torch.tensor([_w1(v[0]) * _w1(v[1]) * _w1(v[2]) for v in VELOCITIES], dtype=DTYPE)
