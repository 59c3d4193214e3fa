"""Host-side index maps of this build's kernels, compiled from the library's own headers with nvcc
into a host program and checked by brute force (no GPU):

* band_row_boxes (csrc/lbm_internal.h): the adjoint's backward step splits the grid's rows into the
  box holding the band's rows, which waits for the immersed-boundary chain, and up to four boxes
  around it, which run beside that chain; every row must lie in exactly one box and every box
  must be non-empty.
* tma_tiles / tma_tile (csrc/lbm_step_tma.cuh): the tensor-copy fed kernel's row tiles cover every
  node 16 <= x < nx - 16 of the rows it runs exactly once; each tile's width is a positive multiple
  of 8 nodes, its copy box [x0 - 8, x0 + 248) starts inside the row on a 16-byte boundary of 16-bit
  values, and the pair reads of its last node stay inside the box's 256 values."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_11856_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "lbm_step_kernels.cuh"
using namespace lbm;

static int check_boxes() {
    long long cases = 0;
    for (int gny = 1; gny <= 9; ++gny)
        for (int gnz = 1; gnz <= 9; ++gnz)
            for (int y0 = 0; y0 < gny; ++y0)
                for (int y1 = y0; y1 < gny; ++y1)
                    for (int z0 = 0; z0 < gnz; ++z0)
                        for (int z1 = z0; z1 < gnz; ++z1) {
                            RowBox band, around[4];
                            const int n = band_row_boxes(gny, gnz, y0, y1, z0, z1, band, around);
                            std::vector<int> hits(gny * gnz, 0);
                            for (int b = -1; b < n; ++b) {
                                const RowBox &r = b < 0 ? band : around[b];
                                if (r.ny < 1 || r.nz < 1 || r.y0 < 0 || r.z0 < 0 || r.y0 + r.ny > gny || r.z0 + r.nz > gnz) {
                                    printf("bad box %d %d | %d %d %d %d\n", gny, gnz, r.y0, r.ny, r.z0, r.nz);
                                    return 1;
                                }
                                for (int z = r.z0; z < r.z0 + r.nz; ++z)
                                    for (int y = r.y0; y < r.y0 + r.ny; ++y) ++hits[y + gny * z];
                            }
                            for (int z = 0; z < gnz; ++z)
                                for (int y = 0; y < gny; ++y) {
                                    const bool in_band = y >= y0 && y <= y1 && z >= z0 && z <= z1;
                                    if (hits[y + gny * z] != 1) { printf("row %d %d hit %d times\n", y, z, hits[y + gny * z]); return 1; }
                                    if (in_band && !(y >= band.y0 && y < band.y0 + band.ny && z >= band.z0 && z < band.z0 + band.nz)) {
                                        printf("band row outside the band box\n");
                                        return 1;
                                    }
                                }
                            ++cases;
                        }
    printf("boxes %lld\n", cases);
    return 0;
}

static int check_tiles() {
    long long cases = 0;
    for (int nx = 40; nx <= 720; nx += 8)
        for (int ny = 1; ny <= 6; ++ny)
            for (int nz = 1; nz <= 5; ++nz)
                for (int inner = 0; inner <= 1; ++inner) {
                    Geometry g{};
                    g.nx = nx; g.ny = ny; g.nz = nz;
                    const TmaTiles T = tma_tiles(g, inner);
                    std::vector<int> hits((size_t)nx * ny * nz, 0);
                    for (long long k = 0; k < T.count; ++k) {
                        int y, z, x0, wt;
                        tma_tile(g, T, k, y, z, x0, wt);
                        if (y < 0 || y >= ny || z < 0 || z >= nz || wt < 8 || wt % 8 || wt > TMA_W || x0 - 8 < 0 ||
                            (x0 - 8) % 8 || x0 + wt > nx - XEDGE || wt + 16 > TMA_SEG) {
                            printf("bad tile nx %d k %lld: y %d z %d x0 %d wt %d\n", nx, k, y, z, x0, wt);
                            return 1;
                        }
                        for (int x = x0; x < x0 + wt; ++x) ++hits[x + (size_t)nx * (y + (size_t)ny * z)];
                    }
                    for (int z = 0; z < nz; ++z)
                        for (int y = 0; y < ny; ++y) {
                            const bool runs = !inner || (y >= 1 && y <= ny - 2 && z >= 1 && z <= nz - 2);
                            for (int x = 0; x < nx; ++x) {
                                const int want = runs && x >= XEDGE && x < nx - XEDGE ? 1 : 0;
                                if (hits[x + (size_t)nx * (y + (size_t)ny * z)] != want) {
                                    printf("node %d %d %d of nx %d hit %d times\n", x, y, z, nx,
                                           hits[x + (size_t)nx * (y + (size_t)ny * z)]);
                                    return 1;
                                }
                            }
                        }
                    ++cases;
                }
    printf("tiles %lld\n", cases);
    return 0;
}

int main() {
    if (check_boxes() || check_tiles()) return 1;
    printf("ok\n");
    return 0;
}
"""


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_row_boxes_and_tensor_copy_tiles(tmp_path):
    exe = nvcc()
    if exe is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "host_tiles.cu"
    src.write_text(PROGRAM)
    binary = tmp_path / "host_tiles"
    # the library's target (its headers use sm_100+ packed FP32 intrinsics); only host code runs
    r = subprocess.run([exe, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(binary)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(binary)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
