"""Benchmark of the fused D3Q27 ACM-MRT + immersed-boundary step on GB300.

Workload: the single-GPU large scene, 1200 x 250 x 840 cells (252M) with ~3.8M procedural
"building" samples at 0.5-cell spacing, inlet u = 0.08 with 1 % seeded noise, outlet,
no-slip ground, free-slip top, periodic z (stand-in for the paper's Fig. 1 / Table 3 scene).
One timed step = one time step of the whole hot path (band moments, interpolation +
penalty, spreading, fused stream + collide over all cells).  The state (27 GB FP32)
is far larger than L2, so no flush is needed between steps.  The K timed steps run in five
timed regions without per-kernel events (value = K steps over their summed time; runs,
median and spread per region); the per-kernel times come from a second, profiled region of
K steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead
(the baseline of this method; there is no other reference implementation).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

BYTES_PER_CELL = {"f32": 216, "f16": 108, "bf16": 108}   # 27 loads + 27 stores per cell update
PAPER_MLUPS = 1200 * 250 * 840 / 1.21 / 1e6                # Table 3, Fig. 1 scene: 1.21 s/step on 4x P40
# DRAM bytes per cell of the main-range kernel from one ncu capture of the current kernel, mean of
# the two AA parities: k_step_main for FP32 (profiles/k_step_main_box_city_480x100x336.md),
# k_step_pair for FP16 (profiles/k_step_pair_box_city_480x100x336.md); absent once a kernel changes
TRAFFIC_PER_CELL = {"f32": 221.3, "f16": 110.3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink every grid axis (testing only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the per-field errors against the stored oracle run")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-models", action="store_true", help="skip the BGK / raw-MRT comparison runs")
    ap.add_argument("--no-tracers", action="store_true", help="skip the smoke-tracer run")
    ap.add_argument("--no-moving", action="store_true", help="skip the rotating-torus run")
    ap.add_argument("--pair-kernel", default="pairs", choices=["pairs", "tma"],
                    help="16-bit storage main range: node pairs loading their own values (default) or fed by tensor copies")
    ap.add_argument("--tracers", type=int, default=4_000_000, help="smoke tracers of the tracer run")
    ap.add_argument("--adjoint-only", action="store_true", help="time only the adjoint workload")
    ap.add_argument("--adjoint-steps", type=int, default=200, help="steps of the adjoint workload")
    ap.add_argument("--adjoint-k", type=int, default=20, help="checkpoint interval of the adjoint workload")
    return ap.parse_args()


def workload(scale):
    nx, ny, nz = (max(8, int(round(n * scale))) for n in (1200, 250, 840))
    n_boxes = max(4, int(round(200 * scale * scale)))
    d = scenes.scene_box_city(nx, ny, nz, n_boxes=n_boxes, with_state=False)
    return d


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(d, steps, block=None):
    """FP64 oracle on a bounded block of the workload: by default the full x-y extent and
    4 cells of z; ``block`` = (x0, nx, y0, ny, nz) picks a smaller box.  The block keeps
    the scene's face types and the samples that fall inside it."""
    import torch
    from oracle.solver import OracleSolver, Problem
    x0, bx, y0, by, bz = block if block is not None else (0, d["nx"], 0, d["ny"], 4)
    z0 = d["nz"] // 2
    X, A = d["samples"], d["area"]
    lo = np.array([x0, y0, z0], dtype=np.float64)
    hi = lo + np.array([bx - 1, by - 1, bz - 1], dtype=np.float64)
    keep = np.all((X >= lo) & (X < hi), axis=1)
    Xs = X[keep] - lo
    p = Problem(bx, by, bz, nu=d["nu"], faces=d["faces"], u_in=d["u_in"], noise=d["noise"], seed=2101)
    o = OracleSolver(p)
    rho, u = scenes.uniform_flow(bx, by, bz, (d["u_in"], 0, 0))
    o.set_state(rho, u)
    if keep.any():
        o.set_solids(Xs, A[keep])
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = bx * by * bz
    return {"value": cells * steps / dt / 1e6, "unit": "MLUPS", "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{bx}x{by}x{bz} block at ({x0},{y0},{z0}) of the same scene ({int(keep.sum())} samples), "
                      f"{steps} steps, FP64"}, dt


REFERENCE_BLOCK = (500, 96, 0, 96, 4)     # one reference-arm step: 36,864 cells near the buildings


def max_over_ranks(x, dist, device):
    """The largest value of x over the ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    d = workload(args.scale)
    blk = REFERENCE_BLOCK if args.scale == 1.0 else None
    for _ in range(args.warmup):
        oracle_sample(d, 1, blk)
    vals, times = [], []
    for _ in range(args.steps):
        cb, dt = oracle_sample(d, 1, blk)
        vals.append(cb["value"])
        times.append(dt)
    value = float(np.mean(vals))
    cb["value"] = value
    line = {"impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"box_city_{d['nx']}x{d['ny']}x{d['nz']}", "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def adjoint_cost(torch, args, dims=None, K=None):
    """Adjoint workload: 128^3 channel, IB sphere r = 12.6 at (40, 64, 64) with 2,000 samples,
    200 steps, loss = mean drag + kinetic energy of the slab 96 <= x < 128, checkpoints every
    20 steps (--adjoint-steps / --adjoint-k change the last two, for small profiling runs).
    ``dims`` = (nx, ny, nz) runs the same channel scaled to that grid (sphere centre at 40/128 of
    the length, radius and sample count scaled with ny, slab the last quarter); ``K`` overrides
    the checkpoint interval.  Reports the adjoint (forward + backward) time against the same
    number of forward steps."""
    from paper_2101_11856_gb300 import Solver
    if dims is None:
        n = max(8, int(round(128 * args.scale))) if args.scale < 1.0 else 128
        dims = (n, n, n)
    nx, ny, nz = dims
    steps, K = args.adjoint_steps, (args.adjoint_k if K is None else K)
    f = ny / 128.0
    count = int(round(2000 * f * f))
    X, A = scenes.fibonacci_sphere((40.0 * nx / 128, ny / 2, nz / 2), 12.6 * f, count)
    rho, u = scenes.uniform_flow(nx, ny, nz, (0.05, 0, 0))
    faces = ("inlet", "outlet", "periodic", "periodic", "periodic", "periodic")
    x0 = int(96 * nx / 128)

    def make():
        s = Solver(nx, ny, nz, 0.01, faces=faces, u_in=0.05, noise=0.01, seed=2101)
        s.set_state(rho, u)
        s.set_solids(X, A)
        return s

    s = make()
    s.step(5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(steps)
    torch.cuda.synchronize()
    fwd = time.perf_counter() - t0
    s.close()
    s = make()
    s.adjoint(2, 1, 1.0, 1.0, x0, nx)     # warm-up (allocations, module load)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L, dcoef, dpos = s.adjoint(steps, K, 1.0, 1.0, x0, nx)
    torch.cuda.synchronize()
    adj = time.perf_counter() - t0
    s.close()
    torch.cuda.empty_cache()
    ok = bool(np.isfinite(L) and np.all(np.isfinite(dcoef)) and np.all(np.isfinite(dpos)))
    N = nx * ny * nz
    return {"workload": f"channel_sphere_{nx}x{ny}x{nz}", "samples": count, "steps": steps, "checkpoint_K": K,
            "state_mb": round(N * 27 * 4 / 1e6, 1),
            "forward_ms": fwd * 1e3, "adjoint_ms": adj * 1e3, "adjoint_over_forward": adj / fwd,
            "adjoint_mlups": N * steps / adj / 1e6, "finite": ok,
            "what": f"lbm_adjoint (forward with checkpoints + segment recompute + backward) vs lbm_step x {steps}"}


def tracer_run(torch, lbm, make, d, args, N, n_int, peak, world, steps):
    """Box city with smoke injected at the inlet: tracers seeded in the emitter slab
    1 <= x < 41, 1 <= y < 121 (all z) and re-injected there.  Reports the whole step with the
    velocity output and the advection, the advection kernel against its algorithmic bytes
    (positions read + written, 2 x 8 corners x 3 velocity components gathered: 216 B per
    tracer) and one density projection on the grid of spacing 2."""
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    P = args.tracers
    lo, hi = (1.0, 1.0, 0.0), (float(min(41, nx - 2)), float(min(121, ny - 2)), float(nz))
    rng = np.random.default_rng(2101)
    X = (np.array(lo) + rng.uniform(0, 1, (P, 3)) * (np.array(hi) - np.array(lo))).astype(np.float32)
    s = make("f32")
    s.set_tracers(X, (lo, hi, 2101))
    del X
    s.step(args.warmup)
    torch.cuda.synchronize()
    ms, kt = timed_steps(s, steps, torch)
    adv_ms = kt["tracer"][0] / max(kt["tracer"][1], 1)
    step_ms = kt["step"][0] / max(kt["step"][1], 1)
    adv_bytes = 216 * P
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dims = lbm.lbm_tracer_dims(s.h, 2)
    grid = torch.empty(dims[2], dims[1], dims[0], device="cuda")
    lbm.lbm_tracer_density(s.h, 2, grid)           # allocates the workspace once
    torch.cuda.synchronize()
    e0.record()
    lbm.lbm_tracer_density(s.h, 2, grid)
    e1.record()
    torch.cuda.synchronize()
    dens_ms = e0.elapsed_time(e1)
    mass = float(grid.double().sum())
    s.close()
    torch.cuda.empty_cache()
    if abs(mass - P) > 1e-4 * P:
        raise RuntimeError(f"tracer density mass {mass} != {P}")
    ach = adv_bytes / (adv_ms * 1e-3) / 1e9
    step_ach = 228 * n_int / (step_ms * 1e-3) / 1e9
    return {"count": P, "emitter": [lo, hi], "mlups": world * N / (ms / steps * 1e-3) / 1e6, "ms_per_step": ms / steps,
            "step_kernel_ms": step_ms,
            "step_kernel_roofline": {"achieved": step_ach, "frac": step_ach / peak, "bytes_per_cell": 228,
                                     "what": "216 B populations + 12 B velocity output"},
            "advect_ms": adv_ms,
            "advect_roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                "bytes_per_tracer": 216},
            "density_ms": dens_ms, "density_grid": list(dims), "density_mass": mass}


def moving_run(torch, lbm, Solver, args, peak, world):
    """Rotating torus (53,280 samples, 400 x 200 x 400, tumbling about x): whole steps with
    the per-step re-pose, re-sort and band rebuild of the moving solid."""
    sc = scenes.scene_rotating_torus()
    nx, ny, nz = sc["nx"], sc["ny"], sc["nz"]
    N = nx * ny * nz
    s = Solver(nx, ny, nz, sc["nu"], faces=sc["faces"])
    s.set_state(sc["rho"], sc["u"])
    s.set_solids(sc["samples"].astype(np.float32), sc["area"].astype(np.float32))
    s.set_motion(sc["motion"])
    s.step(args.warmup)
    torch.cuda.synchronize()
    steps = max(20, args.steps // 2)
    ms, kt = timed_steps(s, steps, torch)
    band = int(lbm.lbm_band_size(s.h))
    torque = s.torque()
    s.close()
    torch.cuda.empty_cache()
    k = kt["step"][0] / max(kt["step"][1], 1)
    n_int = main_cells(nx, ny, nz, sc["faces"])
    ach = 216 * n_int / (k * 1e-3) / 1e9
    if not np.all(np.isfinite(torque)):
        raise RuntimeError("non-finite torque in the rotating-torus run")
    return {"workload": sc["name"], "samples": int(sc["samples"].shape[0]), "band_nodes": band,
            "mlups": world * N / (ms / steps * 1e-3) / 1e6, "ms_per_step": ms / steps,
            "kernel_ms_per_step": {kk: round(v[0] / steps, 4) for kk, v in kt.items() if v[1]},
            "step_kernel_roofline": {"achieved": ach, "frac": ach / peak},
            "torque": list(map(float, torque))}


def main_cells(nx, ny, nz, faces):
    """Nodes one launch of the main step kernel updates: the main range 16 <= x < nx - 16 (16 =
    the edge strip of the face kernel) of every row, or, on a grid with a free-slip face, of the
    rows off the y/z faces (the face rows run with the boundary kernels)."""
    xedge = 16
    if nx < 2 * xedge + 1:
        return 0
    rows = ny * nz
    if "freeslip" in faces:
        rows = max(ny - 2, 0) * max(nz - 2, 0)
    return (nx - 2 * xedge) * rows


def region_steps(solver, steps, torch, regions=5):
    """Time exactly ``steps`` steps without per-kernel profiling, split into ``regions`` timed
    regions of (nearly) equal step counts, each between CUDA events on the solver's stream (torch's
    current stream) with a synchronize on both sides.  Returns (total ms, [(steps, ms) per region])."""
    regions = max(1, min(regions, steps))
    counts = [steps // regions + (1 if r < steps % regions else 0) for r in range(regions)]
    out = []
    for n in counts:
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s0.record()
        solver.step(n)
        s1.record()
        torch.cuda.synchronize()
        out.append((n, s0.elapsed_time(s1)))
    return sum(ms for _, ms in out), out


def run_stats(N, regions, world):
    """MLUPS of every timed region, their median and relative spread (max - min) / median."""
    vals = [world * N * n / (ms * 1e-3) / 1e6 for n, ms in regions]
    med = float(np.median(vals))
    return {"runs": [round(v, 1) for v in vals], "median": med,
            "spread": float((max(vals) - min(vals)) / med) if med > 0 else None}


GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "sphere_channel_256x128x128_100steps.npz")


def precision_vs_oracle(torch, lbm, Solver):
    """Per-field error of each storage against the FP64 oracle on the sphere channel 256 x 128 x 128
    after 100 steps (the oracle's density and velocity at about 110,000 cells, stored by
    tests/golden/make_sphere_channel_golden.py): relative L2 of rho - 1, u_x, u_y, u_z."""
    if not os.path.exists(GOLDEN_C2):
        return None
    z = np.load(GOLDEN_C2)
    idx, rho_o, u_o, meta = z["idx"].astype(np.int64), z["rho"], z["u"], json.loads(str(z["meta"]))
    sc = scenes.scene_sphere_channel(256, 128, 128, radius=meta["radius"], count=meta["count"], u_in=meta["u_in"],
                                     nu=meta["nu"], noise=meta["noise"])
    N = sc["nx"] * sc["ny"] * sc["nz"]
    ti = torch.from_numpy(idx).cuda()
    out = {"workload": sc["name"], "steps": meta["steps"], "cells_compared": int(idx.size),
           "what": "relative L2 over the stored cells against the FP64 oracle"}
    for st in ("f32", "f16", "bf16"):
        g = Solver(sc["nx"], sc["ny"], sc["nz"], sc["nu"], storage=st, faces=sc["faces"], u_in=sc["u_in"],
                   noise=sc["noise"], seed=meta["seed"])
        g.set_state(sc["rho"], sc["u"])
        g.set_solids(sc["samples"].astype(np.float32), sc["area"].astype(np.float32))
        g.step(meta["steps"])
        rho = torch.empty(N, device="cuda")
        u = torch.empty(3, N, device="cuda")
        lbm.lbm_macroscopic(g.h, rho, u)
        g.close()
        rg = rho[ti].double().cpu().numpy()
        ug = u[:, ti].double().cpu().numpy()
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        out[st] = {"rho-1": rel(rg - 1.0, rho_o - 1.0), "u_x": rel(ug[0], u_o[0]), "u_y": rel(ug[1], u_o[1]),
                   "u_z": rel(ug[2], u_o[2]), "rho": rel(rg, rho_o), "u": rel(ug, u_o)}
        del rho, u
    torch.cuda.empty_cache()
    return out


def cpu_model():
    """Host CPU model (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_config_sample(name, steps, dims=None):
    """The FP64 oracle on one configuration, or on a block of it: (MLUPS, seconds, description).
    tgv32: 32^3 periodic Taylor-Green vortex; sphere: the 256 x 128 x 128 sphere channel (a slab
    of it keeps the samples inside); adjoint: the 128^3 channel with its sphere (forward steps)."""
    from oracle.solver import OracleSolver, Problem
    if name == "tgv32":
        sc = scenes.scene_tgv32()
        nx, ny, nz = dims or (32, 32, 32)
        p = Problem(nx, ny, nz, nu=sc["nu"])
        o = OracleSolver(p)
        o.set_state(sc["rho"][:nz, :ny, :nx], sc["u"][:, :nz, :ny, :nx])
    else:
        if name == "sphere":
            sc = scenes.scene_sphere_channel(256, 128, 128, radius=16.0, count=3200, u_in=0.05, nu=0.008)
        else:
            sc = scenes.scene_sphere_channel(128, 128, 128, radius=12.6, count=2000, u_in=0.05, nu=0.01,
                                             center=(40.0, 64.0, 64.0))
        nx, ny, nz = dims or (sc["nx"], sc["ny"], sc["nz"])
        z0 = (sc["nz"] - nz) // 2
        p = Problem(nx, ny, nz, nu=sc["nu"], faces=sc["faces"], u_in=sc["u_in"], noise=sc["noise"], seed=2101)
        o = OracleSolver(p)
        o.set_state(sc["rho"][:nz, :ny, :nx], sc["u"][:, :nz, :ny, :nx])
        X = sc["samples"] - np.array([0.0, 0.0, z0])
        keep = np.all((X >= 0) & (X < np.array([nx - 1, ny - 1, nz - 1])), axis=1)
        if keep.any():
            o.set_solids(X[keep], sc["area"][keep])
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return nx * ny * nz * steps / dt / 1e6, dt, f"{nx}x{ny}x{nz}, {steps} steps"


def cpu_baselines(d, args):
    """The oracle as it stands (FP64, PyTorch CPU) on the host: the benchmark workload's slab with
    all host threads and with one, and bounded samples of the other configurations."""
    import torch
    all_threads = torch.get_num_threads()
    out = {}
    head, _ = oracle_sample(d, 1, (0, d["nx"] // 2, 0, d["ny"], 4))
    torch.set_num_threads(1)
    try:
        one, _ = oracle_sample(d, 1, (2 * d["nx"] // 5, d["nx"] // 8, 0, d["ny"], 4))   # among the buildings
        plan = (("tgv32_100_steps", "tgv32", 100, None, 100, None),
                ("sphere_channel_256x128x128", "sphere", 1, (256, 128, 16), 1, (256, 128, 4)),
                ("adjoint_channel_128^3_forward", "adjoint", 1, (128, 128, 32), 1, (128, 128, 4)))
        for key, name, st_all, dims_all, st_one, dims_one in plan:
            v1, _, s1 = oracle_config_sample(name, st_one, dims_one)
            torch.set_num_threads(all_threads)
            va, _, sa = oracle_config_sample(name, st_all, dims_all)
            torch.set_num_threads(1)
            out[key] = {"cores_all": {"value": va, "sample": sa}, "cores_1": {"value": v1, "sample": s1}}
    finally:
        torch.set_num_threads(all_threads)
    head.update({"cores_all": all_threads, "cpu_model": cpu_model(),
                 "cores_1": {"value": one["value"], "sample": one["sample"]},
                 "configs": out, "unit_note": "MLUPS of the FP64 oracle (cells x steps / s)"})
    return head


def timed_steps(solver, steps, torch):
    from paper_2101_11856_gb300 import lbm
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lbm.lbm_profile(solver.h, True)
    torch.cuda.synchronize()
    s0.record()
    solver.step(steps)
    s1.record()
    torch.cuda.synchronize()
    kt = lbm.lbm_kernel_times(solver.h)
    lbm.lbm_profile(solver.h, False)
    return s0.elapsed_time(s1), kt


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2101_11856_gb300 import Solver, lbm
    lbm.library()
    if args.adjoint_only:
        print(json.dumps({"adjoint": adjoint_cost(torch, args)}))
        return
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if dist is not None:
            dist.barrier()

    d = workload(args.scale)
    nx, ny, nz = d["nx"], d["ny"], d["nz"]
    N = nx * ny * nz
    X = d["samples"].astype(np.float32)
    A = d["area"].astype(np.float32)
    rho0 = torch.ones(N, device="cuda")
    u0 = torch.zeros(3, N, device="cuda")
    u0[0] = d["u_in"]
    peak, peak_kind = measured_peak()

    def make(storage, collision="acm"):
        s = Solver(nx, ny, nz, d["nu"], storage=storage, faces=d["faces"], u_in=d["u_in"], noise=d["noise"], seed=2101,
                   collision=collision)
        s.set_pair_kernel(args.pair_kernel == "tma")
        s.set_state(rho0, u0)
        s.set_solids(X, A)
        return s

    def side_run(storage, collision, steps):
        """Whole-step MLUPS and the main step kernel's roofline for one storage / collision."""
        sx = make(storage, collision)
        sx.step(args.warmup)
        torch.cuda.synchronize()
        msx, ktx = timed_steps(sx, steps, torch)
        kx = ktx["step"][0] / max(ktx["step"][1], 1)
        achx = BYTES_PER_CELL[storage] * n_int / (kx * 1e-3) / 1e9
        massx, _, _ = sx.reductions()
        sx.close()
        torch.cuda.empty_cache()
        if not math.isfinite(massx):
            raise RuntimeError(f"non-finite state in the {storage}/{collision} run")
        return {"mlups": world * N / (msx / steps * 1e-3) / 1e6, "ms_per_step": msx / steps, "step_kernel_ms": kx,
                "roofline": {"bound": "hbm", "achieved": achx, "peak": peak, "unit": "GB/s", "frac": achx / peak,
                             "bytes_per_cell": BYTES_PER_CELL[storage],
                             "traffic": (TRAFFIC_PER_CELL[storage] * n_int
                                         if collision == "acm" and storage in TRAFFIC_PER_CELL else None)}}

    # ---- FP32, device-resident: the headline value -----------------------------------
    s = make("f32")
    band_nodes = int(lbm.lbm_band_size(s.h))
    s.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    with Clocks(local) as clk:
        ms, regions = region_steps(s, args.steps, torch)
    barrier()
    ms_max = max_over_ranks(ms, dist, "cuda" if torch.cuda.is_available() else "cpu")
    ms_step = ms_max / args.steps
    mlups = world * N / (ms_step * 1e-3) / 1e6
    stats = run_stats(N, regions, world)
    # per-kernel times (CUDA events around every launch) from a second region of the same length
    ms_prof, kt = timed_steps(s, args.steps, torch)
    n_int = main_cells(nx, ny, nz, d["faces"])   # cells of one k_step_main launch
    step_ms, step_n = kt["step"]
    k_ms = step_ms / max(step_n, 1)
    achieved = BYTES_PER_CELL["f32"] * n_int / (k_ms * 1e-3) / 1e9
    mass, mom, drag = s.reductions()
    if not (math.isfinite(mass) and np.all(np.isfinite(drag))):
        raise RuntimeError("non-finite state in the benchmark run")
    launches = int(sum(v[1] for v in kt.values()))
    breakdown = {k: round(v[0] / max(v[1], 1), 4) for k, v in kt.items() if v[1]}

    # ---- end to end through the C ABI with host buffers ----------------------------------
    # Batches of 100 steps, each bracketed by the upload of its input fields from pinned host
    # memory and the read-back of its result fields to pinned host memory.  Headline: the
    # asynchronous calls, the next batch's upload and the previous batch's read-back overlapping
    # the steps (every copy inside the timed region; the clock stops when the last read-back
    # landed).  Beside it, the blocking calls with the time of each phase.
    e2e = None
    if not args.no_e2e:
        batch, rounds = 100, 4
        h_rho = torch.ones(N, pin_memory=True)
        h_u = torch.zeros(3, N, pin_memory=True)
        h_u[0] = d["u_in"]
        o_rho = torch.empty(N, pin_memory=True)
        o_u = torch.empty(3, N, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.lbm_set_state_async(s.h, h_rho, h_u)
        for r in range(rounds):
            s.step(batch)
            lbm.lbm_macroscopic_async(s.h, o_rho, o_u)
            if r + 1 < rounds:
                lbm.lbm_set_state_async(s.h, h_rho, h_u)
        lbm.lbm_synchronize(s.h, 600.0)
        dt = time.perf_counter() - t0
        if not bool(torch.isfinite(o_u).all()):
            raise RuntimeError("non-finite fields read back in the end-to-end run")
        phase = np.zeros(3)     # blocking: set_state (H2D + init), steps, macroscopic (+ D2H), seconds
        for _ in range(2):
            ta = time.perf_counter()
            lbm.lbm_set_state(s.h, h_rho, h_u)          # returns after the copy from the host buffers
            tb = time.perf_counter()
            s.step(batch)
            lbm.lbm_synchronize(s.h, 600.0)
            tc = time.perf_counter()
            lbm.lbm_macroscopic(s.h, o_rho, o_u)        # returns after the copy to the host buffers
            phase += (tb - ta, tc - tb, time.perf_counter() - tc)
        e2e = {"value": world * N * batch * rounds / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 16 * N / batch, "d2h_bytes_per_step": 16 * N / batch,
               "steps_per_batch": batch, "batches": rounds, "bytes_per_batch_each_way": 16 * N,
               "what": "per batch: lbm_set_state_async from pinned host rho,u (16 N bytes) + 100 steps + "
                       "lbm_macroscopic_async to pinned host (16 N bytes), copies on the library's copy streams "
                       "overlapping the steps; per-step bytes = batch bytes / 100",
               "serial": {"value": world * N * batch * 2 / phase.sum() / 1e6,
                          "ms_per_batch": {k: round(1e3 * v / 2, 2)
                                           for k, v in zip(("set_state", "steps", "macroscopic"), phase)},
                          "what": "blocking lbm_set_state / lbm_macroscopic around each batch"}}
        del h_rho, h_u, o_rho, o_u
    s.close()
    del s
    torch.cuda.empty_cache()

    # ---- FP16-stored deviations (same workload) ---------------------------------------
    n_side = max(10, args.steps // 2)
    fp16 = None if args.no_fp16 else side_run("f16", "acm", n_side)
    if fp16 is not None:
        fp16["bf16"] = side_run("bf16", "acm", n_side)
        fp16["per_field_error"] = (precision_vs_oracle(torch, lbm, Solver)
                                   if args.scale == 1.0 and not args.no_precision else None)

    # ---- comparison collisions of Sec. 6.1 (same workload, same step structure) -------------
    models = None
    if not args.no_models:
        models = {"acm": {"f32": {"mlups": mlups, "ms_per_step": ms_step, "step_kernel_ms": k_ms,
                                  "roofline": {"achieved": achieved, "frac": achieved / peak}}}}
        if fp16 is not None:
            models["acm"]["f16"] = fp16
        for coll in ("bgk", "raw"):
            models[coll] = {st: side_run(st, coll, n_side) for st in ("f32",) + (() if args.no_fp16 else ("f16",))}

    # ---- smoke tracers in the same flow (velocity output + advection, density projection) ------
    tracers = None
    if not args.no_tracers:
        tracers = tracer_run(torch, lbm, make, d, args, N, n_int, peak, world, n_side)

    moving = None
    if not args.no_moving:
        moving = moving_run(torch, lbm, Solver, args, peak, world)

    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_cost(torch, args)
        if args.scale == 1.0:
            # the same channel on a grid whose state (1.5 GB) is far larger than L2, and the 128^3
            # workload with one segment (every state kept, no recompute)
            adjoint["large_grid"] = adjoint_cost(torch, args, dims=(384, 192, 192))
            adjoint["one_segment"] = adjoint_cost(torch, args, K=args.adjoint_steps)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baselines(d, args)

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": mlups / PAPER_MLUPS,
            "vs_baseline_basis": "paper Table 3, Fig. 1 scene 1200x250x840: 1.21 s/step on 4x Tesla P40 (=208 MLUPS)",
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"box_city_{nx}x{ny}x{nz}", "cells": N, "samples": int(X.shape[0]),
                       "band_nodes": band_nodes,
                       "storage": "f32 deviations, AA in place", "l2": "state 27 GB >> L2, no flush needed",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": TRAFFIC_PER_CELL["f32"] * n_int if TRAFFIC_PER_CELL.get("f32") else None,
                         "kernel": "k_step_main (fused stream+collide, 16 <= x < nx-16 of the rows off the y/z faces)",
                         "cells_per_launch": n_int, "bytes_per_cell": 216,
                         "peak_kind": peak_kind},
            "runs": stats["runs"], "median": stats["median"], "spread": stats["spread"],
            "timing": {"regions": len(regions), "steps_per_region": [n for n, _ in regions],
                       "what": "value = K steps / their summed time over the regions (no per-kernel events); "
                               "runs = MLUPS of each region; kernel times from a separate profiled region of K "
                               f"steps ({ms_prof / args.steps:.3f} ms/step with the events)"},
            "kernel_ms": breakdown,
            "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in kt.items() if v[1]},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "fp16": fp16,
            "collision_models": models,
            "tracers": tracers,
            "moving_solid": moving,
            "adjoint": adjoint,
            "cpu_baseline": cpu,
            "checks": {"mass": mass, "drag": list(map(float, drag))},
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
