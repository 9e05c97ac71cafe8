"""CPU: the multi-rank host logic of bench.py (--gpus N runs N independent
replicas, one per GPU): per-rank seeds, the slowest rank's time as the job time,
whole-job throughput.  Two gloo ranks on the CPU stand in for two GPUs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2311_00921_gb300 import inputs as I  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
        out[rank] = bench.max_over_ranks(ms, dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5


def test_replicas_differ_only_in_seed():
    base = I.WORKLOADS["sphere_yukawa_256k"]
    w0, w1 = bench.replica_workload(base, 0), bench.replica_workload(base, 1)
    assert w0 == base and w1.seed != w0.seed
    assert (w1.n, w1.leaf, w1.rank, w1.kernel) == (w0.n, w0.leaf, w0.rank, w0.kernel)


def test_job_tflops_counts_every_rank():
    one = bench.job_tflops(1, 1e12, 1000.0)
    assert one == pytest.approx(1.0)
    assert bench.job_tflops(4, 1e12, 1000.0) == pytest.approx(4.0)
