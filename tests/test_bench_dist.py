"""The multi-process path of bench.py on CPU (gloo, world size 2): replicas
are timed by the maximum over ranks and the value counts every rank's work;
non-zero ranks of the reference arm exit without output."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    dist.barrier()
    ms_step, value = bench.aggregate_replicas(10.0 + 30.0 * rank, 1000, 5, dist, "cpu")
    out[rank] = (ms_step, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_work():
    port = 29000 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms_step, value = res[rank]
        assert ms_step == pytest.approx(40.0 / 5)          # the slower rank's 40 ms
        assert value == pytest.approx(2 * 1000 / (8e-3) / 1e9)


def test_single_process_aggregation_is_local():
    import bench
    ms_step, value = bench.aggregate_replicas(20.0, 500, 4, None)
    assert ms_step == 5.0 and value == pytest.approx(500 / 5e-3 / 1e9)


def test_reference_arm_nonzero_rank_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env,
                       timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env,
                       timeout=300)
    assert p.returncode == 0
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
