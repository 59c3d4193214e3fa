"""Pins of the oracle's comparison collision models (Sec. 6.1: D3Q27 BGK and raw-moment MRT)
against independent closed forms, special cases and exact viscous decay (no GPU)."""
import itertools
import math

import numpy as np
import pytest
import torch

import scenes
from oracle import collision as col
from oracle.lattice import CF, DTYPE, VELOCITIES
from oracle.solver import OracleSolver, Problem


def random_state(n, seed=0):
    g = torch.Generator().manual_seed(seed)
    rho = 1.0 + 0.05 * (torch.rand(n, generator=g, dtype=DTYPE) - 0.5)
    u = 0.1 * (2 * torch.rand(3, n, generator=g, dtype=DTYPE) - 1)
    f = col.equilibrium(rho, u) * (1.0 + 0.05 * (2 * torch.rand(27, n, generator=g, dtype=DTYPE) - 1))
    F = 1e-3 * (2 * torch.rand(3, n, generator=g, dtype=DTYPE) - 1)
    return f, F


def closed_form_force(u, F):
    """Per axis: g(+-1) = (2u +- 1)/2, g(0) = -2u carries the force; the other axes carry the
    1-D equilibrium factor (written independently of the oracle's matrix solve)."""
    def phi(c, ua):
        return 2 / 3 - ua ** 2 if c == 0 else (1 / 3 + ua ** 2 + c * ua) / 2

    def gam(c, ua):
        return -2 * ua if c == 0 else (2 * ua + c) / 2

    return torch.stack([F[0] * gam(c[0], u[0]) * phi(c[1], u[1]) * phi(c[2], u[2])
                        + F[1] * phi(c[0], u[0]) * gam(c[1], u[1]) * phi(c[2], u[2])
                        + F[2] * phi(c[0], u[0]) * phi(c[1], u[1]) * gam(c[2], u[2]) for c in VELOCITIES])


def raw_direct(f, p, q, r):
    return sum(c[0] ** p * c[1] ** q * c[2] ** r * f[i] for i, c in enumerate(VELOCITIES))


def guo_u(f, F):
    rho = f.sum(0)
    j = torch.einsum("ia,in->an", CF, f)
    return rho, (j + F / 2) / rho


def test_force_distribution_closed_form():
    f, F = random_state(40)
    rho, u = guo_u(f, F)
    assert (col.force_distribution(u, F) - closed_form_force(u, F)).abs().max() < 1e-15


@pytest.mark.parametrize("omega", [0.7, 1.5, 1.95])
def test_bgk_equals_single_rate_moment_relaxation(omega):
    f, F = random_state(50, seed=1)
    rates = {k: omega for k in ("shear", "bulk", "o3", "o4", "o5", "o6")}
    rates["conserved"] = 0.0
    assert (col.collide_bgk(f, F, omega) - col.collide_matrix(f, F, rates)).abs().max() < 1e-14


def test_raw_with_equal_rates_is_bgk():
    f, F = random_state(50, seed=2)
    rates = {k: 1.3 for k in ("shear", "bulk", "o3", "o4", "o5", "o6")}
    rates["conserved"] = 0.0
    assert (col.collide_raw(f, F, rates) - col.collide_bgk(f, F, 1.3)).abs().max() < 1e-14


@pytest.mark.parametrize("model", ["bgk", "raw"])
def test_conservation_and_fixed_point(model):
    f, F = random_state(60, seed=3)
    rates = {"conserved": 0.0, "shear": 1.7, "bulk": 1.1, "o3": 1.3, "o4": 0.9, "o5": 1.45, "o6": 1.05}
    coll = (lambda f_, F_: col.collide_bgk(f_, F_, 1.7)) if model == "bgk" else (lambda f_, F_: col.collide_raw(f_, F_, rates))
    out = coll(f, F)
    assert (out.sum(0) - f.sum(0)).abs().max() < 1e-14
    assert (torch.einsum("ia,in->an", CF, out) - torch.einsum("ia,in->an", CF, f) - F).abs().max() < 1e-14
    rho = f.sum(0)
    u = 0.07 * torch.ones(3, 60, dtype=DTYPE)
    feq = col.equilibrium(rho, u)
    assert (coll(feq, torch.zeros(3, 60, dtype=DTYPE)) - feq).abs().max() < 1e-15


def test_raw_moments_relax_at_their_rates():
    f, F = random_state(30, seed=4)
    rates = {"conserved": 0.0, "shear": 1.7, "bulk": 1.1, "o3": 1.3, "o4": 0.9, "o5": 1.45, "o6": 1.05}
    out = col.collide_raw(f, F, rates)
    rho, u = guo_u(f, F)
    feq = col.equilibrium(rho, u)
    G = closed_form_force(u, F)
    order_rate = {2: rates["shear"], 3: rates["o3"], 4: rates["o4"], 5: rates["o5"], 6: rates["o6"]}
    for p, q, r in itertools.product(range(3), repeat=3):
        if (p, q, r) in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
            continue
        k0, k1 = raw_direct(f, p, q, r), raw_direct(out, p, q, r)
        ke, kg = raw_direct(feq, p, q, r), raw_direct(G, p, q, r)
        w = 0.0 if p + q + r <= 1 else order_rate[p + q + r]
        assert (k1 - (k0 - w * (k0 - ke) + (1 - w / 2) * kg)).abs().max() < 1e-14, (p, q, r)
    neq0 = [raw_direct(f - feq, *e) for e in ((2, 0, 0), (0, 2, 0), (0, 0, 2))]
    g2 = [raw_direct(G, *e) for e in ((2, 0, 0), (0, 2, 0), (0, 0, 2))]
    post = [raw_direct(out - feq, *e) for e in ((2, 0, 0), (0, 2, 0), (0, 0, 2))]
    tr = (1 - rates["bulk"]) * sum(neq0) + (1 - rates["bulk"] / 2) * sum(g2)
    assert (sum(post) - tr).abs().max() < 1e-14


@pytest.mark.parametrize("model", ["bgk", "raw"])
def test_shear_wave_viscosity(model):
    n, A, nu, steps = 32, 1e-4, 0.05, 100
    p = Problem(4, 4, n, nu=nu, collision=model, omega_hi=(1.2, 1.1, 1.0, 0.9))
    s = OracleSolver(p)
    rho, u = scenes.shear_wave(n, A)
    s.set_state(rho[:, :4, :4], u[:, :, :4, :4])
    sinz = torch.sin(2 * math.pi * torch.arange(n, dtype=DTYPE) / n)
    amp = []
    for t in range(steps + 1):
        if t:
            s.step()
        amp.append(float((s.macroscopic()[1][0].mean((1, 2)) * sinz).sum() * 2 / n))
    rate = -np.polyfit(np.arange(steps + 1), np.log(np.abs(amp)), 1)[0] / (2 * math.pi / n) ** 2
    assert abs(rate / nu - 1) < 0.01
