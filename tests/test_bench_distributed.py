"""The N > 1 path of bench.py on CPU with gloo: the max-over-ranks timing reduction across two
ranks, and the reference arm launched by torch.distributed.run with two processes (rank 0
prints the one JSON line, the other rank exits 0 without work).  No GPU."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"


def test_main_kernel_cells():
    """The roofline's cells per main-kernel launch: the main range 16 <= x < nx - 16 of every
    row, or of the rows off the y/z faces on a grid with a free-slip face (those rows run with
    the boundary kernels); no main range below nx = 33."""
    sys.path.insert(0, ROOT)
    import bench
    city = ("inlet", "outlet", "noslip", "freeslip", "periodic", "periodic")
    closed = ("inlet", "outlet", "noslip", "noslip", "periodic", "periodic")
    assert bench.main_cells(1200, 250, 840, city) == 1168 * 248 * 838 == 242738432
    assert bench.main_cells(1200, 250, 840, closed) == 1168 * 250 * 840
    assert bench.main_cells(65, 2, 7, city) == 0            # every row on a face
    assert bench.main_cells(33, 9, 9, closed) == 9 * 9      # one main-range node per row
    assert bench.main_cells(32, 9, 9, closed) == 0          # no main range


def test_run_statistics_and_cpu_samples():
    """The per-region statistics of the headline (MLUPS per region, median, relative spread) and
    one bounded oracle sample of another configuration, on the host."""
    sys.path.insert(0, ROOT)
    import bench
    st = bench.run_stats(1_000_000, [(4, 2.0), (4, 4.0), (4, 2.0)], 1)
    assert st["runs"] == [2000.0, 1000.0, 2000.0] and st["median"] == 2000.0 and abs(st["spread"] - 0.5) < 1e-12
    v, dt, desc = bench.oracle_config_sample("tgv32", 1, (8, 8, 8))
    assert v > 0 and dt > 0 and desc == "8x8x8, 1 steps"
    v, dt, desc = bench.oracle_config_sample("sphere", 1, (24, 12, 6))
    assert v > 0 and desc.startswith("24x12x6")
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
