"""Writes the expected values of the full-size sphere-channel parity test
(tests/test_gpu_sphere_channel.py): the FP64 oracle run of the sphere channel 256 x 128 x 128
(Fibonacci sphere of radius 16 at (64, 64, 64) with 3,200 samples, inlet u = 0.05 with 1 %
seeded noise, outlet, periodic y and z, nu = 0.008, Re = 200) for 100 steps from the uniform
inflow state, and its density and Guo-shifted velocity (Eq. 2) at a fixed set of cells:

* every band node (the 2x2x2 stencil of each sample, Eqs. 6-8),
* the whole inlet plane x = 0 and outlet plane x = 255 (the face rules),
* the planes x = 64 (through the sphere's centre), x = 96 and x = 160 (its wake),
* 20,000 further cells drawn with a seeded generator.

Only ``oracle`` and ``scenes`` are used.  Run from the repository root:
    python tests/golden/make_sphere_channel_golden.py
(about 15 minutes and 20 GB of host memory on 8 cores).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402
from oracle.solver import OracleSolver, Problem  # noqa: E402

OUT = os.path.join(HERE, "sphere_channel_256x128x128_100steps.npz")
STEPS = 100
SEED = 2101


def cell_set(nx, ny, nz, X):
    cells = set()
    base = np.floor(X).astype(np.int64)
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        b = base + off
        cells.update((b[:, 0] + nx * (b[:, 1] + ny * b[:, 2])).tolist())
    y, z = np.meshgrid(np.arange(ny), np.arange(nz), indexing="ij")
    for x in (0, nx - 1, 64, 96, 160):
        cells.update((x + nx * (y + ny * z)).ravel().tolist())
    rng = np.random.default_rng(SEED)
    cells.update(rng.integers(0, nx * ny * nz, 20000).tolist())
    return np.array(sorted(cells), dtype=np.int64)


def main():
    s = scenes.scene_sphere_channel(256, 128, 128, radius=16.0, count=3200, u_in=0.05, nu=0.008)
    nx, ny, nz = s["nx"], s["ny"], s["nz"]
    p = Problem(nx, ny, nz, nu=s["nu"], faces=s["faces"], u_in=s["u_in"], noise=s["noise"], seed=SEED)
    o = OracleSolver(p)
    o.set_state(s["rho"], s["u"])
    o.set_solids(s["samples"], s["area"])
    t0 = time.perf_counter()
    for t in range(STEPS):
        o.step(1)
        if (t + 1) % 10 == 0:
            print(f"step {t + 1}: {time.perf_counter() - t0:.0f} s", flush=True)
    rho, u = (a.numpy() for a in o.macroscopic())
    idx = cell_set(nx, ny, nz, s["samples"])
    meta = dict(scene=s["name"], steps=STEPS, nu=s["nu"], u_in=s["u_in"], noise=s["noise"], seed=SEED,
                radius=16.0, count=3200, faces=list(s["faces"]), cells=int(idx.size),
                drag=[float(v) for v in o.diag["drag"]],
                what="FP64 oracle, rho and Guo-shifted u of the last collision at the listed flat cell indices "
                     "x + nx (y + ny z)")
    np.savez_compressed(OUT, idx=idx.astype(np.int32), rho=rho.reshape(-1)[idx],
                        u=u.reshape(3, -1)[:, idx], meta=json.dumps(meta))
    print(f"wrote {OUT}: {idx.size} cells, drag {meta['drag']}")


if __name__ == "__main__":
    main()
