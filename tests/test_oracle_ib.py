"""Pins of the oracle immersed-boundary stage (Eqs. 6-8) against kernel identities and
brute force (no GPU)."""
import torch

from oracle import ib
from oracle.lattice import DTYPE


def samples(n, shape, seed=0):
    nz, ny, nx = shape
    g = torch.Generator().manual_seed(seed)
    hi = torch.tensor([nx - 1, ny - 1, nz - 1], dtype=DTYPE)
    return torch.rand(n, 3, generator=g, dtype=DTYPE) * (hi - 1e-9)


def test_partition_of_unity_and_first_moment():
    X = samples(500, (9, 8, 7))
    b, K = ib.stencil(X)
    assert (K.sum(1) - 1).abs().max() < 1e-15
    assert (K >= 0).all()
    pos = torch.zeros_like(X)
    for k, d in enumerate(ib.CORNERS):
        pos += K[:, k:k + 1] * (b + torch.tensor(d)).to(DTYPE)
    assert (pos - X).abs().max() < 1e-13


def test_weights_equal_hat_kernel():
    X = samples(200, (6, 6, 6), seed=1)
    b, K = ib.stencil(X)
    for k, d in enumerate(ib.CORNERS):
        node = (b + torch.tensor(d)).to(DTYPE)
        assert (ib.hat(X - node) - K[:, k]).abs().max() < 1e-15


def test_affine_field_interpolated_exactly():
    shape = (7, 6, 9)
    nz, ny, nx = shape
    z, y, x = (t.to(DTYPE) for t in torch.meshgrid(torch.arange(nz), torch.arange(ny), torch.arange(nx),
                                                   indexing="ij"))
    field = 0.3 + 0.1 * x - 0.2 * y + 0.05 * z
    X = samples(300, shape, seed=2)
    expect = 0.3 + 0.1 * X[:, 0] - 0.2 * X[:, 1] + 0.05 * X[:, 2]
    assert (ib.interpolate(field, X) - expect).abs().max() < 1e-14


def test_spread_conserves_total_force():
    shape = (8, 8, 8)
    X = samples(100, shape, seed=3)
    g = torch.randn(3, 100, dtype=DTYPE)
    F = ib.spread_scatter(g, X, shape)
    assert (F.sum((1, 2, 3)) - g.sum(1)).abs().max() < 1e-13


def test_scatter_equals_bruteforce_gather():
    """The paper states that spreading by sample (scatter) is equivalent to Eq. 8's
    per-node sum (gather); brute force over all samples on an 8^3 box."""
    shape = (8, 8, 8)
    X = samples(5, shape, seed=4)
    X[0] = torch.tensor([3.0, 4.0, 2.0], dtype=DTYPE)        # sample exactly on a node
    X[1] = torch.tensor([2.5, 1.0, 6.25], dtype=DTYPE)       # on a cell face
    g = torch.randn(3, 5, dtype=DTYPE)
    a = ib.spread_scatter(g, X, shape)
    b = ib.spread_gather(g, X, shape)
    assert (a - b).abs().max() <= 1e-14 * g.abs().max()


def test_spreading_is_transpose_of_interpolation():
    shape = (6, 7, 8)
    X = samples(40, shape, seed=5)
    phi = torch.randn(*shape, dtype=DTYPE)
    g = torch.randn(40, dtype=DTYPE)
    lhs = (ib.interpolate(phi, X) * g).sum()
    F = ib.spread_scatter(torch.stack([g, g, g]), X, shape)[0]
    rhs = (phi * F).sum()
    assert abs(float(lhs - rhs)) < 1e-12
