"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64 oracle on the same
seeded inputs and compare."""
import numpy as np
import pytest
import torch

from oracle.lattice import VELOCITIES
from oracle.solver import OracleSolver, Problem


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib_solver(**kw):
    from paper_2101_11856_gb300 import Solver
    return Solver(**kw)


def gpu_order():
    """Oracle direction i -> library direction d, matched by velocity vectors."""
    from paper_2101_11856_gb300 import lbm
    lib = {lbm.lbm_velocity(d): d for d in range(27)}
    return [lib[v] for v in VELOCITIES]


def run_pair(nx, ny, nz, nu, steps, rho, u, faces=("periodic",) * 6, forcing=(0.0, 0.0, 0.0), samples=None,
             area=None, u_b=None, storage="f32", u_in=0.0, noise=0.0, seed=2101, inflow_coef=None,
             omega_bulk=1.0, omega_hi=(1.0, 1.0, 1.0, 1.0), oracle_collision=None, collision="acm"):
    """Run both sides; return (gpu solver, oracle solver) after `steps` steps.  ``collision`` is
    the library's model ("acm", "bgk", "raw"); the oracle runs the same model unless
    ``oracle_collision`` names one of its forms explicitly."""
    if oracle_collision is None:
        oracle_collision = {"acm": "factorised", "bgk": "bgk", "raw": "raw"}[collision]
    g = lib_solver(nx=nx, ny=ny, nz=nz, nu=nu, forcing=forcing, storage=storage, faces=faces, u_in=u_in,
                   noise=noise, seed=seed, inflow_coef=inflow_coef, omega_bulk=omega_bulk, omega_hi=omega_hi,
                   collision=collision)
    g.set_state(rho, u)
    o = OracleSolver(Problem(nx, ny, nz, nu=nu, forcing=tuple(forcing), faces=tuple(faces), u_in=u_in, noise=noise,
                             seed=seed, omega_bulk=omega_bulk, omega_hi=tuple(omega_hi), collision=oracle_collision),
                     inflow_coef=inflow_coef)
    o.set_state(rho, u)
    if samples is not None:
        g.set_solids(samples, area, u_b)
        o.set_solids(samples, area, u_b)
    g.step(steps)
    o.step(steps)
    return g, o


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def compare_fields(g, o):
    """(rel L2 of rho, rel L2 of rho - 1, rel L2 of u) between the two sides."""
    rg, ug = g.macroscopic()
    ro, uo = (t.numpy() for t in o.macroscopic())
    return rel_l2(rg, ro), rel_l2(rg - 1.0, ro - 1.0), rel_l2(ug, uo)


def compare_populations(g, o):
    """max |f_gpu - f_oracle| over all populations and cells."""
    fg = g.populations()
    fo = o.populations().numpy()
    order = gpu_order()
    return float(max(np.abs(fg[order[i]] - fo[i]).max() for i in range(27)))
