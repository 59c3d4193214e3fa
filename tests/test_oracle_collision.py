"""Pins of the oracle collision (Eqs. 2, 4, 5) against invariants, textbook special cases
and the mathematics of moment-space relaxation (no GPU).

Each test computes its expectation with code of its own (explicit sums over the 27
velocities), not by calling back into the oracle routine under test.
"""
import itertools

import numpy as np
import pytest
import torch

from oracle import collision as col
from oracle.lattice import CF, DTYPE, VELOCITIES, W

torch.manual_seed(0)


def random_state(n, umax=0.1, spread=0.02, seed=0):
    g = torch.Generator().manual_seed(seed)
    rho = 1.0 + 0.05 * (torch.rand(n, generator=g, dtype=DTYPE) - 0.5)
    u = umax * (2 * torch.rand(3, n, generator=g, dtype=DTYPE) - 1)
    feq = col.equilibrium(rho, u)
    f = feq * (1.0 + spread * (2 * torch.rand(27, n, generator=g, dtype=DTYPE) - 1))
    F = 1e-3 * (2 * torch.rand(3, n, generator=g, dtype=DTYPE) - 1)
    return f, F


def distinct_rates():
    return {"conserved": 0.0, "shear": 1.7, "bulk": 1.1, "o3": 1.3, "o4": 0.9, "o5": 1.45, "o6": 1.05}


def cm_direct(f, u, p, q, r):
    """sum_i (c_ix-u_x)^p (c_iy-u_y)^q (c_iz-u_z)^r f_i, written out over the velocities."""
    out = 0.0
    for i, c in enumerate(VELOCITIES):
        out = out + (c[0] - u[0]) ** p * (c[1] - u[1]) ** q * (c[2] - u[2]) ** r * f[i]
    return out


def guo_u(f, F):
    rho = f.sum(0)
    j = torch.stack([sum(VELOCITIES[i][a] * f[i] for i in range(27)) for a in range(3)])
    return rho, (j + F / 2) / rho


def test_equilibrium_rest_weights():
    rho = torch.tensor([1.3], dtype=DTYPE)
    feq = col.equilibrium(rho, torch.zeros(3, 1, dtype=DTYPE))
    assert torch.allclose(feq[:, 0], 1.3 * W, atol=1e-15)


def test_equilibrium_moments():
    f, _ = random_state(50)
    rho = f.sum(0)
    u = 0.1 * (2 * torch.rand(3, 50, dtype=DTYPE) - 1)
    feq = col.equilibrium(rho, u)
    assert torch.allclose(feq.sum(0), rho, atol=1e-15)
    assert torch.allclose(torch.einsum("ia,in->an", CF, feq), rho * u, atol=1e-15)
    P = torch.einsum("ia,ib,in->abn", CF, CF, feq)
    expect = rho * (u[:, None] * u[None, :] + torch.eye(3, dtype=DTYPE)[:, :, None] / 3)
    assert torch.allclose(P, expect, atol=1e-15)
    # central moments of the discrete equilibrium are rho * m_p m_q m_r, m = (1, 0, 1/3)
    m = (1.0, 0.0, 1.0 / 3.0)
    for p, q, r in itertools.product(range(3), repeat=3):
        assert torch.allclose(cm_direct(feq, u, p, q, r), rho * m[p] * m[q] * m[r], atol=1e-15)


@pytest.mark.parametrize("path", ["matrix", "factorised"])
def test_equilibrium_is_fixed_point(path):
    f, _ = random_state(20)
    rho = f.sum(0)
    u = 0.08 * (2 * torch.rand(3, 20, dtype=DTYPE) - 1)
    feq = col.equilibrium(rho, u)
    coll = col.collide_matrix if path == "matrix" else col.collide_factorised
    out = coll(feq, torch.zeros(3, 20, dtype=DTYPE), distinct_rates())
    assert torch.allclose(out, feq, atol=1e-15)


def test_matrix_and_factorised_paths_agree():
    f, F = random_state(200, spread=0.05)
    rates = distinct_rates()
    a = col.collide_matrix(f, F, rates)
    b = col.collide_factorised(f, F, rates)
    assert (a - b).abs().max() < 1e-13


@pytest.mark.parametrize("path", ["matrix", "factorised"])
def test_mass_and_momentum_conservation(path):
    f, F = random_state(100, spread=0.05)
    coll = col.collide_matrix if path == "matrix" else col.collide_factorised
    out = coll(f, F, distinct_rates())
    assert (out.sum(0) - f.sum(0)).abs().max() < 1e-14
    j0 = torch.einsum("ia,in->an", CF, f)
    j1 = torch.einsum("ia,in->an", CF, out)
    assert (j1 - (j0 + F)).abs().max() < 1e-14


def force_distribution(u, F):
    """M^-1 R^F in closed form from per-axis raw-moment matching.

    Per axis the force factor is the 1-D distribution g with sum g = 0, sum (c-u) g = 1,
    sum (c-u)^2 g = 0, i.e. g(+-1) = (2u +- 1)/2, g(0) = -2u; the other axes carry the
    1-D equilibrium factor phi (central moments 1, 0, 1/3).
    """
    def phi(c, ua):
        return 2 / 3 - ua ** 2 if c == 0 else (1 / 3 + ua ** 2 + c * ua) / 2

    def gam(c, ua):
        return -2 * ua if c == 0 else (2 * ua + c) / 2

    out = []
    for c in VELOCITIES:
        out.append(F[0] * gam(c[0], u[0]) * phi(c[1], u[1]) * phi(c[2], u[2])
                   + F[1] * phi(c[0], u[0]) * gam(c[1], u[1]) * phi(c[2], u[2])
                   + F[2] * phi(c[0], u[0]) * phi(c[1], u[1]) * gam(c[2], u[2]))
    return torch.stack(out)


@pytest.mark.parametrize("omega", [0.6, 1.0, 1.9])
def test_single_rate_reduces_to_bgk_with_guo_forcing(omega):
    f, F = random_state(60, spread=0.05)
    rates = {"conserved": 0.0, "shear": omega, "bulk": omega, "o3": omega, "o4": omega,
             "o5": omega, "o6": omega}
    rho, u = guo_u(f, F)
    feq = col.equilibrium(rho, u)
    G = force_distribution(u, F)
    # textbook Guo force-term moments: sum G = 0, sum c G = F, sum cc G = uF + Fu
    assert G.sum(0).abs().max() < 1e-16
    assert (torch.einsum("ia,in->an", CF, G) - F).abs().max() < 1e-16
    P = torch.einsum("ia,ib,in->abn", CF, CF, G)
    assert (P - (u[:, None] * F[None, :] + F[:, None] * u[None, :])).abs().max() < 1e-16
    expect = f - omega * (f - feq) + (1 - omega / 2) * G
    for coll in (col.collide_matrix, col.collide_factorised):
        assert (coll(f, F, rates) - expect).abs().max() < 1e-14


def test_unit_rates_give_equilibrium_plus_half_force():
    f, F = random_state(40, spread=0.05)
    rates = {"conserved": 0.0, "shear": 1.0, "bulk": 1.0, "o3": 1.0, "o4": 1.0, "o5": 1.0, "o6": 1.0}
    rho, u = guo_u(f, F)
    expect = col.equilibrium(rho, u) + 0.5 * force_distribution(u, F)
    assert (col.collide_factorised(f, F, rates) - expect).abs().max() < 1e-14


def test_each_moment_relaxes_at_its_own_rate():
    """Central moments of the output, taken directly, follow
    k' = k - w (k - k_eq) + (1 - w/2) R^F with the rate of the moment's group; the
    diagonal second-order moments via the trace (omega_b) and deviators (omega_s)."""
    f, F = random_state(30, spread=0.05)
    rates = distinct_rates()
    out = col.collide_factorised(f, F, rates)
    rho, u = guo_u(f, F)
    m = (1.0, 0.0, 1.0 / 3.0)
    order_rate = {2: rates["shear"], 3: rates["o3"], 4: rates["o4"], 5: rates["o5"], 6: rates["o6"]}
    for p, q, r in itertools.product(range(3), repeat=3):
        if (p, q, r) in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
            continue
        k0 = cm_direct(f, u, p, q, r)
        k1 = cm_direct(out, u, p, q, r)
        keq = rho * m[p] * m[q] * m[r]
        rf = F[0] * (p == 1) * m[q] * m[r] + F[1] * (q == 1) * m[p] * m[r] + F[2] * (r == 1) * m[p] * m[q]
        w = 0.0 if p + q + r <= 1 else order_rate[p + q + r]
        assert (k1 - (k0 - w * (k0 - keq) + (1 - w / 2) * rf)).abs().max() < 1e-14, (p, q, r)
    neq0 = [cm_direct(f, u, *e) - rho / 3 for e in ((2, 0, 0), (0, 2, 0), (0, 0, 2))]
    neq1 = [cm_direct(out, u, *e) - rho / 3 for e in ((2, 0, 0), (0, 2, 0), (0, 0, 2))]
    tr0, tr1 = sum(neq0), sum(neq1)
    assert (tr1 - (1 - rates["bulk"]) * tr0).abs().max() < 1e-14
    for a, b in ((0, 1), (0, 2)):
        assert ((neq1[a] - neq1[b]) - (1 - rates["shear"]) * (neq0[a] - neq0[b])).abs().max() < 1e-14


def test_within_group_basis_mixing_leaves_operator_unchanged():
    """Any invertible recombination of basis rows within one rate group gives the same
    Omega (D is a multiple of the identity on every group), e.g. a non-orthogonal basis."""
    f, F = random_state(25, spread=0.05)
    rates = distinct_rates()
    rho, u = guo_u(f, F)
    M = col.moment_matrix(u)
    D = col.rate_vector(rates)
    groups = [g for (_, g, _) in col.BASIS]
    B = torch.zeros(27, 27, dtype=DTYPE)
    gen = torch.Generator().manual_seed(3)
    for gname in set(groups):
        idx = [k for k, g in enumerate(groups) if g == gname]
        blk = torch.eye(len(idx), dtype=DTYPE) + 0.4 * torch.rand(len(idx), len(idx), generator=gen, dtype=DTYPE)
        for a, ia in enumerate(idx):
            for b, ib in enumerate(idx):
                B[ia, ib] = blk[a, b]
    M2 = B @ M
    feq = col.equilibrium(rho, u)
    RF2 = col.force_moments(F) @ B.T
    rhs = -D * torch.einsum("nki,in->nk", M2, f - feq) + (1 - D / 2) * RF2
    out2 = f + torch.linalg.solve(M2, rhs.unsqueeze(-1)).squeeze(-1).T
    assert (out2 - col.collide_matrix(f, F, rates)).abs().max() < 1e-13
