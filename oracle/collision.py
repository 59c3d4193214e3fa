"""Central-moment MRT collision with Guo-style body forcing (Eqs. 2, 4, 5).

ORACLE -- test infrastructure only.

Eq. 5 relaxes the distributions in a moment space, Omega = -M^-1 D M (f - f_eq), with a
27x27 projection M and a diagonal matrix D of rates; Eq. 4 adds the external-force term
G.  The paper gives the structure but defers the ACM-MRT basis, equilibrium and
adaptive high-order rates to its supplement (not available).  Readings used here:

* M(u) is the central-moment matrix: row (p,q,r), p,q,r in {0,1,2}, entry
  (c_ix - u_x)^p (c_iy - u_y)^q (c_iz - u_z)^r, the moment monomials the paper's
  Table 2 shows (up to u_x^2 u_y^2 u_z^2).  The three diagonal second-order rows are
  recombined into the trace (200+020+002) and two deviators (200-020, 200-002).
* u is the Guo-shifted velocity u = (sum_i c_i f_i + F/2) / rho (Eq. 2 plus the
  half-force shift of Guo forcing).
* f_eq is the product-form discrete Maxwellian whose central moments are
  rho * m_p m_q m_r with m = (1, 0, 1/3).
* Rates: shear omega_s = 1 / (3 nu + 1/2) on the off-diagonal second-order moments and
  the two deviators (so nu = c_s^2 (1/omega_s - 1/2)); omega_b on the trace; one
  constant rate per order for orders 3, 4, 5, 6 (the adaptive rule is not available --
  parity unpinned for it); conserved moments (orders 0, 1) have rate 0.
* Forcing: the central moments of the force term are
  R^F_pqr = F_x [p=1] m_q m_r + F_y [q=1] m_p m_r + F_z [r=1] m_p m_q, applied as
  (I - D/2) R^F, i.e. f_post = f + M^-1 [ -D (M f - M f_eq) + (I - D/2) R^F ].

``collide_matrix`` evaluates that expression literally, building M(u) per node and
solving with it; ``collide_factorised`` applies the same operator through the
tensor-product structure of M(u) (one 3x3 transform per axis).  The two are pinned
against each other and against conservation laws, fixed points, textbook special cases
and exact viscous decay in ``tests/test_oracle_collision.py``.
"""
from __future__ import annotations

import torch

from .lattice import CF, DTYPE, VELOCITIES

# Central moments of the continuous Maxwellian (per axis, c_s^2 = 1/3): m_0, m_1, m_2.
M1D = (1.0, 0.0, 1.0 / 3.0)

# Moment-space basis rows: (label, rate group, [(coefficient, (p, q, r)), ...]).
BASIS = (
    [("000", "conserved", [(1.0, (0, 0, 0))]),
     ("100", "conserved", [(1.0, (1, 0, 0))]),
     ("010", "conserved", [(1.0, (0, 1, 0))]),
     ("001", "conserved", [(1.0, (0, 0, 1))]),
     ("110", "shear", [(1.0, (1, 1, 0))]),
     ("101", "shear", [(1.0, (1, 0, 1))]),
     ("011", "shear", [(1.0, (0, 1, 1))]),
     ("200-020", "shear", [(1.0, (2, 0, 0)), (-1.0, (0, 2, 0))]),
     ("200-002", "shear", [(1.0, (2, 0, 0)), (-1.0, (0, 0, 2))]),
     ("200+020+002", "bulk", [(1.0, (2, 0, 0)), (1.0, (0, 2, 0)), (1.0, (0, 0, 2))])]
    + [(f"{p}{q}{r}", "o3", [(1.0, (p, q, r))])
       for (p, q, r) in ((2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1), (1, 0, 2), (0, 1, 2), (1, 1, 1))]
    + [(f"{p}{q}{r}", "o4", [(1.0, (p, q, r))])
       for (p, q, r) in ((2, 2, 0), (2, 0, 2), (0, 2, 2), (2, 1, 1), (1, 2, 1), (1, 1, 2))]
    + [(f"{p}{q}{r}", "o5", [(1.0, (p, q, r))]) for (p, q, r) in ((2, 2, 1), (2, 1, 2), (1, 2, 2))]
    + [("222", "o6", [(1.0, (2, 2, 2))])]
)
assert len(BASIS) == 27


def omega_shear(nu: float) -> float:
    """Shear relaxation rate from the kinematic viscosity, nu = c_s^2 (1/omega - 1/2)."""
    return 1.0 / (3.0 * nu + 0.5)


def relaxation_rates(nu: float, omega_bulk: float = 1.0, omega_hi=(1.0, 1.0, 1.0, 1.0)) -> dict:
    """Rate of every group of Eq. 5's diagonal D (low orders from nu, high orders given)."""
    return {"conserved": 0.0, "shear": omega_shear(nu), "bulk": float(omega_bulk),
            "o3": float(omega_hi[0]), "o4": float(omega_hi[1]),
            "o5": float(omega_hi[2]), "o6": float(omega_hi[3])}


def density_momentum(f: torch.Tensor):
    """rho = sum_i f_i and j = sum_i c_i f_i (Eq. 2); f has shape (27, ...)."""
    rho = f.sum(0)
    j = torch.einsum("ia,i...->a...", CF, f)
    return rho, j


def guo_velocity(rho, j, F):
    """Velocity with the half-force shift of Guo forcing: u = (j + F/2) / rho."""
    return (j + 0.5 * F) / rho


def _phi(c: int, ua: torch.Tensor) -> torch.Tensor:
    # 1-D discrete distribution with central moments (1, 0, 1/3) about ua
    if c == 0:
        return 2.0 / 3.0 - ua * ua
    return (1.0 / 3.0 + ua * ua + c * ua) / 2.0


def equilibrium(rho: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """Product-form equilibrium f_eq_i = rho * prod_a phi(c_ia, u_a); shape (27, ...)."""
    return torch.stack([rho * _phi(c[0], u[0]) * _phi(c[1], u[1]) * _phi(c[2], u[2])
                        for c in VELOCITIES])


def moment_matrix(u: torch.Tensor) -> torch.Tensor:
    """Explicit M(u) of Eq. 5 for every node: u (3, N) -> (N, 27, 27)."""
    n = u.shape[1]
    rel = CF.T[:, None, :] - u[:, :, None]          # (3, N, 27): c_ia - u_a
    powers = [torch.ones_like(rel), rel, rel * rel]
    M = torch.zeros(n, 27, 27, dtype=DTYPE)
    for row, (_, _, terms) in enumerate(BASIS):
        for coef, (p, q, r) in terms:
            M[:, row, :] += coef * powers[p][0] * powers[q][1] * powers[r][2]
    return M


def force_moments(F: torch.Tensor) -> torch.Tensor:
    """R^F in the basis rows: F (3, N) -> (N, 27)."""
    out = torch.zeros(F.shape[1], 27, dtype=DTYPE)
    m = M1D
    for row, (_, _, terms) in enumerate(BASIS):
        for coef, (p, q, r) in terms:
            val = (F[0] * (p == 1) * m[q] * m[r] + F[1] * (q == 1) * m[p] * m[r]
                   + F[2] * (r == 1) * m[p] * m[q])
            out[:, row] += coef * val
    return out


def rate_vector(rates: dict) -> torch.Tensor:
    """Diagonal of D in the basis-row order."""
    return torch.tensor([rates[g] for (_, g, _) in BASIS], dtype=DTYPE)


def collide_matrix(f: torch.Tensor, F: torch.Tensor, rates: dict) -> torch.Tensor:
    """f_post = f + Omega + G with Omega = -M^-1 D M (f - f_eq) and G = M^-1 (I - D/2) R^F.

    Literal form of Eqs. 4-5: builds the 27x27 M(u) at every node and solves with it.
    f: (27, *S) pre-collision (streamed) distributions; F: (3, *S) total force.
    """
    shape = f.shape[1:]
    f2 = f.reshape(27, -1)
    F2 = F.reshape(3, -1)
    rho, j = density_momentum(f2)
    u = guo_velocity(rho, j, F2)
    feq = equilibrium(rho, u)
    M = moment_matrix(u)
    D = rate_vector(rates)
    m_neq = torch.einsum("nki,in->nk", M, f2 - feq)
    rhs = -D * m_neq + (1.0 - 0.5 * D) * force_moments(F2)
    df = torch.linalg.solve(M, rhs.unsqueeze(-1)).squeeze(-1)       # (N, 27)
    return (f2 + df.T).reshape(27, *shape)


# ---- tensor-product form ------------------------------------------------------------

_GRID = [(c[0] + 1, c[1] + 1, c[2] + 1) for c in VELOCITIES]


def _to_grid(f2: torch.Tensor) -> torch.Tensor:
    g = torch.zeros(3, 3, 3, f2.shape[1], dtype=f2.dtype)
    for i, (a, b, c) in enumerate(_GRID):
        g[a, b, c] = f2[i]
    return g


def _from_grid(g: torch.Tensor) -> torch.Tensor:
    return torch.stack([g[a, b, c] for (a, b, c) in _GRID])


def _axis_transform(ua: torch.Tensor) -> torch.Tensor:
    """Per-axis factor of M(u): T[n, p, a] = (a - 1 - u_n)^p, shape (N, 3, 3)."""
    c = torch.tensor([-1.0, 0.0, 1.0], dtype=DTYPE)
    rel = c[None, :] - ua[:, None]
    return torch.stack([torch.ones_like(rel), rel, rel * rel], dim=1)


def central_moments(f2: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """kappa[p, q, r, n] = sum_i (c_ix-u_x)^p (c_iy-u_y)^q (c_iz-u_z)^r f_i (tensor form)."""
    Tx, Ty, Tz = (_axis_transform(u[a]) for a in range(3))
    return torch.einsum("npa,nqb,nrc,abcn->pqrn", Tx, Ty, Tz, _to_grid(f2))


def from_central_moments(kappa: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """Inverse of ``central_moments``: one 3x3 inverse per axis and node."""
    Ix, Iy, Iz = (torch.linalg.inv(_axis_transform(u[a])) for a in range(3))
    return _from_grid(torch.einsum("nap,nbq,ncr,pqrn->abcn", Ix, Iy, Iz, kappa))


def collide_factorised(f: torch.Tensor, F: torch.Tensor, rates: dict) -> torch.Tensor:
    """Same operator as ``collide_matrix`` through the per-axis central-moment transform."""
    shape = f.shape[1:]
    f2 = f.reshape(27, -1)
    F2 = F.reshape(3, -1)
    rho, j = density_momentum(f2)
    u = guo_velocity(rho, j, F2)
    k = central_moments(f2, u)
    m = M1D
    out = torch.empty_like(k)
    order_rate = {3: rates["o3"], 4: rates["o4"], 5: rates["o5"], 6: rates["o6"]}
    ws, wb = rates["shear"], rates["bulk"]
    for p in range(3):
        for q in range(3):
            for r in range(3):
                keq = rho * (m[p] * m[q] * m[r])
                rf = F2[0] * (p == 1) * m[q] * m[r] + F2[1] * (q == 1) * m[p] * m[r] \
                    + F2[2] * (r == 1) * m[p] * m[q]
                o = p + q + r
                if o <= 1:
                    w = rates["conserved"]
                elif (p, q, r) in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
                    continue                      # diagonal second order: below
                elif o == 2:
                    w = ws
                else:
                    w = order_rate[o]
                out[p, q, r] = k[p, q, r] - w * (k[p, q, r] - keq) + (1.0 - 0.5 * w) * rf
    # diagonal second order: trace relaxed with omega_b, deviators with omega_s
    a = k[2, 0, 0] - rho * m[2]
    b = k[0, 2, 0] - rho * m[2]
    c = k[0, 0, 2] - rho * m[2]
    tr = (1.0 - wb) * (a + b + c)
    d1 = (1.0 - ws) * (a - b)
    d2 = (1.0 - ws) * (a - c)
    out[2, 0, 0] = rho * m[2] + (tr + d1 + d2) / 3.0
    out[0, 2, 0] = rho * m[2] + (tr - 2.0 * d1 + d2) / 3.0
    out[0, 0, 2] = rho * m[2] + (tr + d1 - 2.0 * d2) / 3.0
    return from_central_moments(out, u).reshape(27, *shape)


# ---- comparison collision models (Sec. 6.1: D3Q27 BGK and raw-moment MRT) -------------
# The paper compares ACM-MRT with the D3Q27 BGK and RM-MRT models under the same
# streaming, forcing and boundary treatment.  Readings: BGK relaxes every population with
# the shear rate towards the product equilibrium and adds the force term G = M(u)^-1 R^F
# with the factor (1 - omega/2) (Guo); RM-MRT is Eq. 5 with the moment matrix taken at u = 0
# (raw moments c_x^p c_y^q c_z^r, same rows and rate groups as above), equilibrium M f_eq and
# force moments M G.

def force_distribution(u: torch.Tensor, F: torch.Tensor) -> torch.Tensor:
    """Discrete force term G = M(u)^-1 R^F of Eq. 4 at every node: u, F (3, N) -> (27, N)."""
    G = torch.linalg.solve(moment_matrix(u), force_moments(F).unsqueeze(-1)).squeeze(-1)
    return G.T


def collide_bgk(f: torch.Tensor, F: torch.Tensor, omega: float) -> torch.Tensor:
    """Single-relaxation-time (BGK) collision with Guo forcing:
    f_post = f - omega (f - f_eq(rho, u)) + (1 - omega/2) G, u = (j + F/2)/rho."""
    shape = f.shape[1:]
    f2 = f.reshape(27, -1)
    F2 = F.reshape(3, -1)
    rho, j = density_momentum(f2)
    u = guo_velocity(rho, j, F2)
    out = f2 - omega * (f2 - equilibrium(rho, u)) + (1.0 - 0.5 * omega) * force_distribution(u, F2)
    return out.reshape(27, *shape)


def collide_raw(f: torch.Tensor, F: torch.Tensor, rates: dict) -> torch.Tensor:
    """Raw-moment MRT: Eq. 5 with M = M(0) (u-independent raw moments)."""
    shape = f.shape[1:]
    f2 = f.reshape(27, -1)
    F2 = F.reshape(3, -1)
    rho, j = density_momentum(f2)
    u = guo_velocity(rho, j, F2)
    M0 = moment_matrix(torch.zeros(3, 1, dtype=DTYPE))[0]
    D = rate_vector(rates)
    m_neq = M0 @ (f2 - equilibrium(rho, u))
    rf = M0 @ force_distribution(u, F2)
    rhs = -D[:, None] * m_neq + (1.0 - 0.5 * D)[:, None] * rf
    return (f2 + torch.linalg.solve(M0, rhs)).reshape(27, *shape)
