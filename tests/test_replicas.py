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


def test_reference_arm_prints_its_contract_line():
    # bench.py --impl reference times the oracle on the host cores: one JSON line with the
    # metric of the GPU arm, the cpu_baseline it describes and an e2e block with no copies
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, cwd=root, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["metric"].startswith("H_eff sigma") and d["unit"] == "TFLOP/s"
    assert d["config"]["workload"] and d["dtype"] == "f64" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
