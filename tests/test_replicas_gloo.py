"""Multi-rank path of bench.py on CPU: two gloo ranks run independent replicas;
the job's rate is every rank's points over the slowest rank's time, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import torch
import torch.distributed as td
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    td.init_process_group("gloo", rank=rank, world_size=world)

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        td.all_reduce(t, op=td.ReduceOp.MAX)
        return t.item()

    # rank r took 100 + 50 r ms for 10 steps of 1000 points each
    ms_step, value = bench.replica_rate(100.0 + 50.0 * rank, 10, 1000, world, reduce_max)
    pts = workloads.unit_gaussian(64, bench.replica_seed(6, rank))
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), ms=ms_step, value=value, pts=pts)
    td.barrier()
    td.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0, r1 = (np.load(tmp_path / f"r{r}.npz") for r in (0, 1))
    for r in (r0, r1):
        assert float(r["ms"]) == 15.0                      # slowest rank: 150 ms / 10 steps
        assert abs(float(r["value"]) - 2000 / 0.015) < 1e-6  # both ranks' points
    assert not np.array_equal(r0["pts"], r1["pts"])        # independent replicas


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    """Rank 0 of the reference arm prints one JSON line with the keys of the
    benchmark contract, naming the same workload as the library's arm."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1
    base = bench.headline_config()
    assert {k: d["config"][k] for k in base} == base
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["sample"] == d["config"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_host_cpu_list_parsing_and_fallback():
    """The end-to-end leg allocates its pinned buffers from the GPU's local
    host cores: sysfs cpu lists parse to sets, and without a GPU (or where
    the topology is not exposed) no affinity change is asked for."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench._cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._cpulist("5") == {5}
    assert bench._cpulist("") == set()
    if not torch.cuda.is_available():
        assert bench._near_gpu_cpus(0) is None
