"""The bench's multi-GPU form is replicas (no data-path collective): two gloo ranks on CPU
check the max-over-ranks timing and the whole-job throughput it reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed 100 + 50 r ms over 5 steps of 2e9 flops each
    ms, tflops = bench.replica_throughput(100.0 + 50.0 * rank, 5, 2e9, world, "cpu")
    q.put((rank, ms, tflops))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, tflops in got:
        assert ms == pytest.approx(150.0 / 5)                       # the slowest rank decides
        assert tflops == pytest.approx(2 * 2e9 / (30e-3) / 1e12)    # both replicas' work


def test_replica_throughput_single_process():
    import bench
    ms, tflops = bench.replica_throughput(40.0, 4, 1e9, 1)
    assert ms == 10.0 and tflops == pytest.approx(0.1)
