"""Multi-rank host logic of the benchmark on CPU: world size 2 over gloo.
The path does not exchange data between ranks (each rank relaxes its own
copy of the workload); the only collective is the max over ranks of the
timed region."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert out[0] == out[1] == 2.5


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def _run_bench(args, env_extra):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], cwd=root, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    # the reference arm times the FP64 oracle on the host cores: one JSON line
    # with the keys of the benchmark contract and the same metric and unit as
    # the GPU arm
    import json
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "relaxation particle-iterations/s" and d["unit"] == "particle-iterations/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # a bounded crop of the vehicle shell: 1/16 of its 19.2 M
    # generated particles, the same workload as the GPU arm's headline
    assert "vehicle" in d["config"]["workload"] and "smallest x" in d["config"]["sample"]
    assert 1.1e6 < d["config"]["particles"] < 1.3e6


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_cpu_baseline_leg_times_the_oracle_on_the_cores_and_on_one_thread():
    import bench
    import oracle
    from paper_2501_03056_gb300 import workloads as W
    before = oracle.get_threads()
    out = bench.cpu_baseline_leg(W.cube_workload(), "sphere_torus")     # whole bodies, one iteration
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] == before
    one = out["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and one["cores_over_one"] > 0
    assert oracle.get_threads() == before                               # the thread count is restored
