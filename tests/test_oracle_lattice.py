"""Pins of the oracle's D3Q27 lattice and noise generator against closed forms and
published test vectors (no GPU)."""
import os

import numpy as np
import torch

from oracle.lattice import C, CF, OPPOSITE, VELOCITIES, W
from oracle.noise import inlet_noise, splitmix64, uniform_pm1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_velocity_set_is_d3q27():
    # every velocity lands on a neighbouring node, all 27 distinct (Eq. 1)
    assert len(set(VELOCITIES)) == 27
    assert all(max(abs(c) for c in v) <= 1 for v in VELOCITIES)
    assert VELOCITIES[0] == (0, 0, 0)
    for i, j in enumerate(OPPOSITE):
        assert tuple(-c for c in VELOCITIES[i]) == VELOCITIES[j]
    # opposite pairs adjacent
    for k in range(1, 27, 2):
        assert OPPOSITE[k] == k + 1


def test_weights_closed_form_and_isotropy():
    norm = C.abs().sum(1)
    expect = {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}
    for i in range(27):
        assert abs(float(W[i]) - expect[int(norm[i])]) < 1e-16
    assert abs(float(W.sum()) - 1.0) < 1e-15
    assert torch.allclose(W @ CF, torch.zeros(3, dtype=W.dtype), atol=1e-16)
    second = torch.einsum("i,ia,ib->ab", W, CF, CF)
    assert torch.allclose(second, torch.eye(3, dtype=W.dtype) / 3, atol=1e-16)
    # fourth-order isotropy: sum w cx^4 = 3 cs^4, sum w cx^2 cy^2 = cs^4
    assert abs(float((W * CF[:, 0] ** 4).sum()) - 1 / 3) < 1e-15
    assert abs(float((W * CF[:, 0] ** 2 * CF[:, 1] ** 2).sum()) - 1 / 9) < 1e-15


def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if not l.startswith("#")]
    for seed, n, val in rows:
        out = splitmix64(int(seed), np.array([int(n)], dtype=np.uint64))[0]
        assert int(out) == int(val, 16)


def test_inlet_noise_range_and_counter():
    xi = inlet_noise(2101, 5, 7, 3)
    assert xi.shape == (3, 7)
    assert (xi >= -1).all() and (xi < 1).all()
    # counter of node (y=4, z=2) at t=5 is (5*7 + 4)*3 + 2
    assert xi[2, 4] == uniform_pm1(2101, np.array([(5 * 7 + 4) * 3 + 2], dtype=np.uint64))[0]
    # roughly uniform
    big = inlet_noise(1, 1, 200, 200)
    assert abs(big.mean()) < 0.02 and abs(big.var() - 1 / 3) < 0.02
