"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): runs with more
than one GPU are independent replicas, timed by the slowest rank, and the whole-job
rate counts every rank's points; only rank 0 runs the reference arm."""
import os
import socket
import subprocess
import sys
import textwrap

from conftest import ROOT

CHILD = textwrap.dedent("""
    import os, sys
    sys.path.insert(0, os.environ["BENCH_ROOT"])
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    rank, ws = dist.get_rank(), dist.get_world_size()
    slowest = bench.max_over_ranks(1.5 + rank, ws)     # rank 1 is the slower one
    assert slowest == 2.5, slowest
    # replicas: every rank streams its own 1e9 points; the job counts all of them
    assert abs(bench.job_rate(1e9, ws, slowest) - 2 * 1e9 / 2.5 / 1e9) < 1e-12
    if rank == 1:
        class A:
            n = 1000
        assert bench.run_reference(A(), ws, rank) is None  # returns before any work
    dist.barrier()
    dist.destroy_process_group()
    print("rank", rank, "ok")
""")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_replicas_aggregate_with_gloo():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank), BENCH_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    for rank, (p, out) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, out
        assert f"rank {rank} ok" in out


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_rate(1e9, 1, 1.25) == 0.8


def test_committed_stream_profile_is_readable():
    """The ncu summary that bench.py reads for `traffic` parses: a 16-hex-digit hash
    of the kernel sources and a DRAM bytes-per-point figure near the 8 bytes the
    float64 stream must read."""
    sys.path.insert(0, ROOT)
    import bench
    kv = bench.profile_summary(os.path.join(ROOT, "profiles", "k_stream_xwidth_f64.md"))
    h = kv["kernel sources sha256[:16]"]
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    assert 8.0 <= float(kv["dram bytes per point"]) < 8.5
