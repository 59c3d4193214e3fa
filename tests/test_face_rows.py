"""The row index of the face-row kernels (grids with a free-slip face): face_rows / face_row
(csrc/lbm_internal.h) enumerate exactly the rows (y, z) on a y or z face, each once, and
face_grid (csrc/lbm_step_kernels.cuh) folds any row count into a grid whose y extent stays
within 65535.  Compiled from the library's own headers with nvcc into a host program and
checked by brute force; no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_11856_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <set>
#include <utility>
#include "lbm_step_kernels.cuh"
using namespace lbm;

int main() {
    long long checked = 0;
    for (int ny = 1; ny <= 40; ++ny)
        for (int nz = 1; nz <= 40; ++nz) {
            Geometry g{};
            g.nx = 70; g.ny = ny; g.nz = nz;
            std::set<std::pair<int, int>> seen;
            const long long R = face_rows(g);
            for (long long r = 0; r < R; ++r) {
                int y = -1, z = -1;
                face_row(g, r, y, z);
                if (y < 0 || y >= ny || z < 0 || z >= nz) { printf("out of range %d %d %lld\n", ny, nz, r); return 1; }
                const bool inner = y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2;
                if (inner) { printf("inner row %d %d %lld\n", ny, nz, r); return 1; }
                if (!seen.insert({y, z}).second) { printf("duplicate %d %d %lld\n", ny, nz, r); return 1; }
            }
            long long want = 0;
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y) want += !(y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2);
            if ((long long)seen.size() != want) { printf("missing rows %d %d\n", ny, nz); return 1; }
            ++checked;
        }
    const long long counts[] = {1, 2, 65534, 65535, 65536, 131070, 131071, 262140, 1000003};
    for (long long n : counts) {
        const dim3 d = face_grid(2, n);
        if (d.x != 2 || d.y < 1 || d.y > 65535 || d.z < 1 || (long long)d.y * d.z < n ||
            (long long)d.y * (d.z - 1) >= n) { printf("fold %lld -> %u %u\n", n, d.y, d.z); return 1; }
    }
    printf("ok %lld\n", checked);
    return 0;
}
"""


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_face_row_map_and_grid_fold(tmp_path):
    exe = nvcc()
    if exe is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "face_rows.cu"
    src.write_text(PROGRAM)
    binary = tmp_path / "face_rows"
    # the library's target (its headers use sm_100+ packed FP32 intrinsics); only host code runs
    r = subprocess.run([exe, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(binary)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(binary)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.startswith("ok 1600"), out.stdout + out.stderr
